"""CPU oracle of the PASTIS hot path: plain, slow, single-threaded C behind ctypes.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import it; the product package never does, and shares no code
with it.  Parity unpinned (definitions of this oracle, not fixed by the paper): the
x-drop pruning order and the symmetrization of A S A^T.
"""
