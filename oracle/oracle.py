"""ctypes front end of the C oracle (oracle/pastis_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by the
CPU-baseline leg of bench.py, never by the product package.  The record dtypes below
mirror the structs declared in pastis_oracle.c and nothing else.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pastis_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

CAND_DTYPE = np.dtype([("i", "<i4"), ("j", "<i4"), ("count", "<u4"),
                       ("qpos", "<u2", (2,)), ("tpos", "<u2", (2,))])
ALN_DTYPE = np.dtype([("score", "<i4"), ("qb", "<u2"), ("qe", "<u2"), ("tb", "<u2"),
                      ("te", "<u2"), ("ident", "<u2"), ("cols", "<u2"),
                      ("seed_used", "u1"), ("passes", "u1"), ("pad", "<u2")])
EDGE_DTYPE = np.dtype([("i", "<i4"), ("j", "<i4"), ("ident", "<u2"), ("cols", "<u2"),
                       ("score", "<i4"), ("weight", "<f4")])
assert CAND_DTYPE.itemsize == 20 and ALN_DTYPE.itemsize == 20 and EDGE_DTYPE.itemsize == 20

SW, XD, SW_SCORE, SW_FILTERED, XD_FILTERED = 0, 1, 2, 3, 4

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, no vector intrinsics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            L.or_encode.restype = i64
            L.or_encode.argtypes = [P, i64, P]
            L.or_kmers.restype = i64
            L.or_kmers.argtypes = [P, P, i32, i32, P, P, P]
            L.or_subkmers.restype = ctypes.c_int
            L.or_subkmers.argtypes = [P, i64, i32, i32, P, P, P]
            L.or_candidates.restype = ctypes.c_int
            L.or_candidates.argtypes = [P, P, P, i32, i32, i32, P, i32,
                                        ctypes.POINTER(P), ctypes.POINTER(i64)]
            L.or_align_pairs.restype = ctypes.c_int
            L.or_align_pairs.argtypes = [P, P, P, i64, P, i32, i32, i32, i32, i32, i32, i32,
                                         P, ctypes.POINTER(i64)]
            L.or_filter.restype = i64
            L.or_filter.argtypes = [P, P, P, i64, i32, i32, P]
            L.or_ns_edges.restype = i64
            L.or_ns_edges.argtypes = [P, P, P, i64, P]
            L.or_components.restype = ctypes.c_int
            L.or_components.argtypes = [i32, P, i64, P]
            L.or_free.restype = None
            L.or_free.argtypes = [P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class InvalidResidue(ValueError):
    pass


def encode(ascii: np.ndarray) -> np.ndarray:
    """Residue letters -> codes 0..23 (Sec. V-B).  Raises InvalidResidue."""
    a = np.ascontiguousarray(ascii, dtype=np.uint8)
    out = np.empty_like(a)
    bad = lib().or_encode(_ptr(a), a.size, _ptr(out))
    if bad >= 0:
        raise InvalidResidue(f"byte {bad} ({a[bad]!r}) is not a residue letter")
    return out


def kmers(codes: np.ndarray, offsets: np.ndarray, k: int):
    """Rows of A (Sec. IV-A): (row_ptr, code, pos), codes ascending per row."""
    c = np.ascontiguousarray(codes, dtype=np.uint8)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    n = o.size - 1
    cap = max(1, int(c.size))
    row_ptr = np.zeros(n + 1, np.int64)
    code = np.zeros(cap, np.uint32)
    pos = np.zeros(cap, np.uint16)
    nnz = lib().or_kmers(_ptr(c), _ptr(o), n, k, _ptr(row_ptr), _ptr(code), _ptr(pos))
    return row_ptr, code[:nnz].copy(), pos[:nnz].copy()


def subkmers(roots: np.ndarray, k: int, m: int, matrix: np.ndarray):
    """Rows of S (Sec. IV-B): [n, m+1] codes and distances, identity first."""
    r = np.ascontiguousarray(roots, dtype=np.uint32)
    mat = np.ascontiguousarray(matrix, dtype=np.int8)
    codes = np.zeros((r.size, m + 1), np.uint32)
    dist = np.zeros((r.size, m + 1), np.int32)
    if lib().or_subkmers(_ptr(r), r.size, k, m, _ptr(mat), _ptr(codes), _ptr(dist)) != 0:
        raise ValueError("invalid k or m")
    return codes, dist


def candidates(row_ptr, code, pos, k: int, m: int, matrix, min_shared: int = 1) -> np.ndarray:
    """Candidate pairs i < j with count and seeds (Sec. IV-A, IV-C)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cd = np.ascontiguousarray(code, dtype=np.uint32)
    ps = np.ascontiguousarray(pos, dtype=np.uint16)
    mat = np.ascontiguousarray(matrix, dtype=np.int8)
    out = ctypes.c_void_p()
    nout = ctypes.c_int64()
    rc = lib().or_candidates(_ptr(rp), _ptr(cd), _ptr(ps), rp.size - 1, k, m, _ptr(mat),
                             min_shared, ctypes.byref(out), ctypes.byref(nout))
    if rc != 0:
        raise ValueError("oracle candidates failed")
    n = nout.value
    res = np.zeros(n, CAND_DTYPE)
    if n:
        ctypes.memmove(res.ctypes.data, out.value, n * CAND_DTYPE.itemsize)
    lib().or_free(out)
    return res


def align_pairs(codes, offsets, pairs, matrix, gap_open=11, gap_extend=1, mode=SW,
                xdrop=49, k=6, ani=30, cov=70):
    """One alignment record per candidate (Sec. IV-E); returns (records, cells)."""
    c = np.ascontiguousarray(codes, dtype=np.uint8)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    p = np.ascontiguousarray(pairs, dtype=CAND_DTYPE)
    mat = np.ascontiguousarray(matrix, dtype=np.int8)
    out = np.zeros(p.size, ALN_DTYPE)
    cells = ctypes.c_int64(0)
    lib().or_align_pairs(_ptr(c), _ptr(o), _ptr(p), p.size, _ptr(mat), gap_open, gap_extend,
                         mode, xdrop, k, ani, cov, _ptr(out), ctypes.byref(cells))
    return out, cells.value


def filter_edges(offsets, pairs, alns, ani=30, cov=70) -> np.ndarray:
    """Edges that pass the ANI/coverage filter (Sec. IV-F), in pair order."""
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    p = np.ascontiguousarray(pairs, dtype=CAND_DTYPE)
    a = np.ascontiguousarray(alns, dtype=ALN_DTYPE)
    out = np.zeros(max(1, p.size), EDGE_DTYPE)
    ne = lib().or_filter(_ptr(o), _ptr(p), _ptr(a), p.size, ani, cov, _ptr(out))
    return out[:ne].copy()


def ns_edges(offsets, pairs, alns) -> np.ndarray:
    """Edges weighted by the normalized score (Sec. VI-B, NS): every pair with a positive
    score, weight = score / shorter length in float32."""
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    p = np.ascontiguousarray(pairs, dtype=CAND_DTYPE)
    a = np.ascontiguousarray(alns, dtype=ALN_DTYPE)
    out = np.zeros(max(1, p.size), EDGE_DTYPE)
    ne = lib().or_ns_edges(_ptr(o), _ptr(p), _ptr(a), p.size, _ptr(out))
    return out[:ne].copy()


def components(n, edges) -> np.ndarray:
    """Connected components (Sec. VI-B): label = smallest vertex of the component."""
    e = np.ascontiguousarray(edges, dtype=EDGE_DTYPE)
    lab = np.zeros(max(1, n), np.int32)
    if lib().or_components(int(n), _ptr(e), e.size, _ptr(lab)) != 0:
        raise ValueError("edge endpoint out of range")
    return lab[:n].copy()


def weighted_precision_recall(labels, families):
    """Weighted precision and recall of a clustering against reference families (the
    measures of protein clustering studies the paper uses, Sec. VI-B): precision = sum
    over clusters of the largest family overlap / N; recall = sum over families of the
    largest cluster overlap / N."""
    labels = np.asarray(labels, dtype=np.int64)
    families = np.asarray(families, dtype=np.int64)
    n = labels.size
    if n == 0:
        return 1.0, 1.0
    pairs = np.stack([labels, families], axis=1)
    uniq, counts = np.unique(pairs, axis=0, return_counts=True)
    best_c = {}
    best_f = {}
    for (c, f), k in zip(uniq.tolist(), counts.tolist()):
        best_c[c] = max(best_c.get(c, 0), k)
        best_f[f] = max(best_f.get(f, 0), k)
    return sum(best_c.values()) / n, sum(best_f.values()) / n


def run(ascii, offsets, matrix, k=6, m=0, min_shared=1, mode=SW, xdrop=49, gap_open=11,
        gap_extend=1, ani=30, cov=70):
    """The whole path a1..a10 on the CPU; returns a dict of every intermediate."""
    codes = encode(ascii)
    row_ptr, code, pos = kmers(codes, offsets, k)
    cands = candidates(row_ptr, code, pos, k, m, matrix, min_shared)
    alns, cells = align_pairs(codes, offsets, cands, matrix, gap_open, gap_extend, mode,
                              xdrop, k, ani, cov)
    edges = filter_edges(offsets, cands, alns, ani, cov)
    return dict(codes=codes, row_ptr=row_ptr, code=code, pos=pos, cands=cands, alns=alns,
                cells=cells, edges=edges)
