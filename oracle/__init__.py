"""CPU oracle of the PASTIS hot path: plain, slow, single-threaded C behind ctypes.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import it; the product package never does, and shares no code
with it.  Two readings are definitions the paper does not give (the x-drop pruning
order, Sec. IV-E, and the symmetrization of A S A^T, Sec. VI-A); both are pinned by
cases worked out by hand (tests/golden/) and by brute force, like every other step.
"""
