"""GB300 (sm_103a) implementation of the PASTIS hot path (Selvitopi et al., SC20).

k-mer matrix A -> semiring SpGEMM candidates (A A^T or A S A^T) -> Smith-Waterman /
x-drop alignment -> ANI/coverage similarity filter, all in hand-written CUDA behind the
C ABI of include/pastis.h.  `pastis` is the thin Python binding of that library.
"""
from . import pastis
from .pastis import (ALN_DTYPE, CAND_DTYPE, EDGE_DTYPE, SW, SW_FILTERED, SW_SCORE, XD, XD_DEFAULT_PER_WARP, XD_FILTERED, AlignPlan, Context, KMat, Params, PastisError,
                     PROBE_KINDS, align_pairs, autotune_sw, autotune_xd, build_kmers, encode, filter_edges, overlap_spgemm,
                     probe_int_throughput, run,
                     substitute_kmers, to_records)
