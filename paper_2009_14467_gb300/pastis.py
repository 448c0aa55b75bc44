"""Python binding of libpastis (include/pastis.h): argument marshalling only.

Every step of the path runs in the library's CUDA kernels; this module moves torch
device pointers and the current CUDA stream across the C ABI, checks status codes and
allocates the caller-owned output buffers with torch.  It never computes a result on
the CPU: if the library is missing, loading it raises.
"""
import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

ALPHABET = "ARNDCQEGHILKMFPSTWYVBZX*"
SW, XD, SW_SCORE, SW_FILTERED, XD_FILTERED = 0, 1, 2, 3, 4
SW_BINS, SW_BIN_WIDTH, SW_MAX_EXTRA = 64, 32, 2     # pass-1 layout per query-length bin
SW_INT32 = 3                                        # a layout value: the bin's pairs in 32-bit lanes
XD_DEFAULT_PER_WARP = 4                             # x-drop extensions per warp in 16-bit lanes

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "INVALID_RESIDUE", 3: "CAPACITY", 4: "OUT_OF_MEMORY",
          5: "CUDA", 6: "TIMEOUT", 7: "UNSUPPORTED", 8: "INTERNAL"}
OK, ERR_CAPACITY = 0, 3

# record layouts of include/pastis.h
CAND_DTYPE = np.dtype([("i", "<i4"), ("j", "<i4"), ("count", "<u4"),
                       ("qpos", "<u2", (2,)), ("tpos", "<u2", (2,))])
ALN_DTYPE = np.dtype([("score", "<i4"), ("qb", "<u2"), ("qe", "<u2"), ("tb", "<u2"),
                      ("te", "<u2"), ("ident", "<u2"), ("cols", "<u2"),
                      ("seed_used", "u1"), ("passes", "u1"), ("reserved", "<u2")])
EDGE_DTYPE = np.dtype([("i", "<i4"), ("j", "<i4"), ("ident", "<u2"), ("cols", "<u2"),
                       ("score", "<i4"), ("weight", "<f4")])
REC_BYTES = 20


class PastisError(RuntimeError):
    def __init__(self, call, status, extra=""):
        self.status = status
        super().__init__(f"{call}: {STATUS.get(status, status)} {extra}".strip())


class c_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("m_subs", ctypes.c_int32), ("min_shared", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("xdrop", ctypes.c_int32), ("gap_open", ctypes.c_int32),
                ("gap_extend", ctypes.c_int32), ("ani_min_pct", ctypes.c_int32),
                ("cov_min_pct", ctypes.c_int32), ("matrix", ctypes.c_int8 * 576)]


class c_kmat(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("k", ctypes.c_int32), ("capacity", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("row_code", ctypes.c_void_p),
                ("row_pos", ctypes.c_void_p), ("col_ptr", ctypes.c_void_p), ("col_seq", ctypes.c_void_p),
                ("col_pos", ctypes.c_void_p)]


@dataclass
class Params:
    """pastis_params: the method's parameters (Sec. VI defaults)."""
    matrix: np.ndarray
    k: int = 6
    m_subs: int = 0
    min_shared: int = 1
    mode: int = SW
    xdrop: int = 49
    gap_open: int = 11
    gap_extend: int = 1
    ani_min_pct: int = 30
    cov_min_pct: int = 70

    def c(self) -> c_params:
        p = c_params()
        for f in ("k", "m_subs", "min_shared", "mode", "xdrop", "gap_open", "gap_extend",
                  "ani_min_pct", "cov_min_pct"):
            setattr(p, f, int(getattr(self, f)))
        m = np.ascontiguousarray(self.matrix, dtype=np.int8).reshape(-1)
        if m.size != 576:
            raise ValueError("the substitution matrix must be 24x24")
        ctypes.memmove(p.matrix, m.ctypes.data, 576)
        return p


_lock = threading.Lock()
_lib = None


def lib():
    """Loads libpastis.so (building it first if needed).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                path = _build.build()
            L = ctypes.CDLL(path)
            P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            sigs = {
                "pastis_ctx_create": [ctypes.POINTER(P), ctypes.c_int, P],
                "pastis_ctx_destroy": [P],
                "pastis_ctx_forget": [P],
                "pastis_encode": [P, P, i64, P, ctypes.POINTER(i64)],
                "pastis_kmat_sizes": [i32, i64, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)],
                "pastis_build_kmers": [P, P, P, i32, i32, ctypes.POINTER(c_kmat), ctypes.POINTER(i64)],
                "pastis_substitute_kmers": [P, P, i64, ctypes.POINTER(c_params), P, P],
                "pastis_overlap_spgemm": [P, ctypes.POINTER(c_kmat), ctypes.POINTER(c_params), P, i64,
                                          ctypes.POINTER(i64)],
                "pastis_overlap_spgemm_rows": [P, ctypes.POINTER(c_kmat), ctypes.POINTER(c_params), i32, i32, P,
                                               i64, ctypes.POINTER(i64)],
                "pastis_align_pairs": [P, P, P, i32, P, i64, ctypes.POINTER(c_params), P, P],
                "pastis_filter_edges": [P, P, i32, P, P, i64, ctypes.POINTER(c_params), P, i64,
                                        ctypes.POINTER(i64)],
            }
            for name, args in sigs.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int32
            L.pastis_status_string.argtypes = [ctypes.c_int32]
            L.pastis_status_string.restype = ctypes.c_char_p
            L.pastis_ctx_workspace_bytes.argtypes = [P]
            L.pastis_ctx_workspace_bytes.restype = i64
            L.pastis_ctx_launch_count.argtypes = [P]
            L.pastis_ctx_launch_count.restype = i64
            L.pastis_ctx_profile.argtypes = [P, ctypes.c_int]
            L.pastis_ctx_profile.restype = ctypes.c_int32
            L.pastis_ctx_profile_read.argtypes = [P, ctypes.c_char_p, ctypes.c_int32]
            L.pastis_ctx_profile_read.restype = ctypes.c_int32
            L.pastis_ctx_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.c_int32]
            L.pastis_ctx_stats.restype = ctypes.c_int32
            _lib = L
    return _lib


def _check(name, st, extra=""):
    if st != OK:
        raise PastisError(name, st, extra)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None and t.numel() > 0 else 0)


class Context:
    """A pastis_ctx on a CUDA device, enqueuing on the torch stream current at creation
    (or the given one).  Owns the library's workspace until closed."""

    def __init__(self, device=0, stream=None):
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check("pastis_ctx_create", lib().pastis_ctx_create(
            ctypes.byref(h), self.device.index or 0, ctypes.c_void_p(self.stream.cuda_stream)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().pastis_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return int(lib().pastis_ctx_launch_count(self.h))

    def forget(self):
        """pastis_ctx_forget: drop the kept AS matrix and the kept product, so the next
        call computes them again."""
        _check("pastis_ctx_forget", lib().pastis_ctx_forget(self.h))

    @property
    def workspace_bytes(self) -> int:
        return int(lib().pastis_ctx_workspace_bytes(self.h))

    def profile(self, enable: bool = True):
        """Per-kernel CUDA-event timing inside the library (see pastis_ctx_profile)."""
        _check("pastis_ctx_profile", lib().pastis_ctx_profile(self.h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kernel name: (launches, total ms)} since profiling was enabled."""
        buf = ctypes.create_string_buffer(1 << 16)
        n = lib().pastis_ctx_profile_read(self.h, buf, len(buf))
        out = {}
        for ln in buf.raw[:n].decode().splitlines():
            name, cnt, ms = ln.split()
            out[name] = (int(cnt), float(ms))
        return out

    def stats(self) -> dict:
        """pastis_ctx_stats: overlap-product work counted while profiling was on."""
        v = (ctypes.c_int64 * 4)()
        _check("pastis_ctx_stats", lib().pastis_ctx_stats(self.h, v, 4))
        return {"spgemm_products": v[0], "spgemm_left_entries": v[1], "spgemm_records": v[2],
                "sort_element_passes": v[3]}

    def sw_layout(self) -> np.ndarray:
        """pastis_sw_layout_get: extra pass-1 stripes per query-length bin (uint8[64])."""
        _layout_sigs()
        out = np.zeros(SW_BINS, np.uint8)
        _check("pastis_sw_layout_get", lib().pastis_sw_layout_get(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_sw_layout(self, extra=None):
        """pastis_sw_layout_set (None: the default layout)."""
        _layout_sigs()
        if extra is None:
            _check("pastis_sw_layout_set", lib().pastis_sw_layout_set(self.h, None))
            return
        a = np.ascontiguousarray(extra, dtype=np.uint8)
        if a.shape != (SW_BINS,):
            raise ValueError(f"a layout has {SW_BINS} entries")
        _check("pastis_sw_layout_set", lib().pastis_sw_layout_set(self.h, a.ctypes.data_as(ctypes.c_void_p)))

    def xd_layout(self) -> int:
        """pastis_xd_layout_get: x-drop extensions per warp in 16-bit lanes (0: 32-bit lanes)."""
        _layout_sigs()
        return int(lib().pastis_xd_layout_get(self.h))

    def set_xd_layout(self, per_warp: int = XD_DEFAULT_PER_WARP):
        """pastis_xd_layout_set: 1, 2 or 4 extensions per warp in 16-bit lanes, 0 for 32-bit lanes."""
        _layout_sigs()
        _check("pastis_xd_layout_set", lib().pastis_xd_layout_set(self.h, int(per_warp)))


@dataclass
class KMat:
    """The caller-owned device arrays of pastis_kmat."""
    n_rows: int
    k: int
    capacity: int
    nnz: int
    row_ptr: torch.Tensor
    row_code: torch.Tensor
    row_pos: torch.Tensor
    col_ptr: torch.Tensor
    col_seq: torch.Tensor
    col_pos: torch.Tensor

    def c(self) -> c_kmat:
        m = c_kmat()
        m.n_rows, m.k, m.capacity, m.nnz = self.n_rows, self.k, self.capacity, self.nnz
        for f in ("row_ptr", "row_code", "row_pos", "col_ptr", "col_seq", "col_pos"):
            setattr(m, f, _ptr(getattr(self, f)).value)
        return m


def encode(ctx: Context, ascii_dev: torch.Tensor, out: torch.Tensor = None) -> torch.Tensor:
    """pastis_encode: uint8 letters (device) -> uint8 codes 0..23."""
    assert ascii_dev.dtype == torch.uint8 and ascii_dev.is_cuda
    out = torch.empty_like(ascii_dev) if out is None else out
    bad = ctypes.c_int64(-1)
    st = lib().pastis_encode(ctx.h, _ptr(ascii_dev), ascii_dev.numel(), _ptr(out), ctypes.byref(bad))
    _check("pastis_encode", st, f"(first bad byte at {bad.value})" if st == 2 else "")
    return out


def kmat_alloc(n: int, total_residues: int, k: int, device) -> KMat:
    cap, cpl = ctypes.c_int64(), ctypes.c_int64()
    _check("pastis_kmat_sizes", lib().pastis_kmat_sizes(n, total_residues, k, ctypes.byref(cap),
                                                        ctypes.byref(cpl)))
    c = max(1, cap.value)
    return KMat(n, k, cap.value, 0,
                torch.empty(n + 1, dtype=torch.int64, device=device),
                torch.empty(c, dtype=torch.int32, device=device),      # uint32 codes, int32 storage
                torch.empty(c, dtype=torch.int16, device=device),      # uint16 positions
                torch.empty(cpl.value, dtype=torch.int32, device=device),
                torch.empty(c, dtype=torch.int32, device=device),
                torch.empty(c, dtype=torch.int16, device=device))


def build_kmers(ctx: Context, codes: torch.Tensor, offsets: torch.Tensor, k: int, A: KMat = None) -> KMat:
    """pastis_build_kmers: A in CSR and CSC (Sec. IV-A)."""
    n = offsets.numel() - 1
    if A is None:
        A = kmat_alloc(n, codes.numel(), k, codes.device)
    cm = A.c()
    nnz = ctypes.c_int64()
    _check("pastis_build_kmers", lib().pastis_build_kmers(ctx.h, _ptr(codes), _ptr(offsets), n, k,
                                                          ctypes.byref(cm), ctypes.byref(nnz)))
    A.nnz = nnz.value
    return A


def substitute_kmers(ctx: Context, roots: torch.Tensor, params: Params):
    """pastis_substitute_kmers: rows of S, [n, m+1] codes (int32 storage) and distances."""
    n = roots.numel()
    m = params.m_subs
    code = torch.empty((n, m + 1), dtype=torch.int32, device=roots.device)
    dist = torch.empty((n, m + 1), dtype=torch.int32, device=roots.device)
    p = params.c()
    _check("pastis_substitute_kmers", lib().pastis_substitute_kmers(ctx.h, _ptr(roots), n, ctypes.byref(p),
                                                                    _ptr(code), _ptr(dist)))
    return code, dist


def overlap_spgemm(ctx: Context, A: KMat, params: Params, capacity: int = 0, rows=None) -> torch.Tensor:
    """pastis_overlap_spgemm (or, with rows=(i0, i1), pastis_overlap_spgemm_rows): candidate
    records (uint8 [n, 20]) sorted by (i, j)."""
    p = params.c()
    cm = A.c()
    nout = ctypes.c_int64()
    r0, r1 = (0, A.n_rows) if rows is None else (int(rows[0]), int(rows[1]))

    def call(buf, cap):
        return lib().pastis_overlap_spgemm_rows(ctx.h, ctypes.byref(cm), ctypes.byref(p), r0, r1, _ptr(buf),
                                                cap, ctypes.byref(nout))

    out = torch.empty((max(capacity, 1), REC_BYTES), dtype=torch.uint8, device=A.row_ptr.device)
    st = call(out, capacity)
    if st == ERR_CAPACITY:
        out = torch.empty((max(nout.value, 1), REC_BYTES), dtype=torch.uint8, device=A.row_ptr.device)
        st = call(out, nout.value)
    _check("pastis_overlap_spgemm", st)
    return out[:nout.value]


def align_pairs(ctx: Context, codes: torch.Tensor, offsets: torch.Tensor, pairs: torch.Tensor,
                params: Params, cells: torch.Tensor = None, out: torch.Tensor = None) -> torch.Tensor:
    """pastis_align_pairs: one alignment record (uint8 [n, 20]) per candidate."""
    n = pairs.shape[0]
    out = torch.empty((max(n, 1), REC_BYTES), dtype=torch.uint8, device=codes.device) if out is None else out
    p = params.c()
    _check("pastis_align_pairs", lib().pastis_align_pairs(ctx.h, _ptr(codes), _ptr(offsets), offsets.numel() - 1,
                                                          _ptr(pairs), n, ctypes.byref(p), _ptr(out),
                                                          _ptr(cells)))
    return out[:n]


def _layout_sigs():
    L = lib()
    if not getattr(L, "_layout_sigs", False):
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.pastis_sw_layout_set.argtypes = [P, P]
        L.pastis_sw_layout_set.restype = i32
        L.pastis_sw_layout_get.argtypes = [P, P]
        L.pastis_sw_layout_get.restype = i32
        L.pastis_xd_layout_set.argtypes = [P, i32]
        L.pastis_xd_layout_set.restype = i32
        L.pastis_xd_layout_get.argtypes = [P]
        L.pastis_xd_layout_get.restype = i32
        L.pastis_autotune_xd.argtypes = [P, P, P, i32, P, P, i32, P, i64, ctypes.POINTER(c_params), i32, P, P]
        L.pastis_autotune_xd.restype = i32
        L.pastis_autotune_sw.argtypes = [P, P, P, i32, P, P, i32, P, i64, ctypes.POINTER(c_params), i32, P, P]
        L.pastis_autotune_sw.restype = i32
        L._layout_sigs = True
    return L


def autotune_sw(ctx: Context, codes: torch.Tensor, offsets: torch.Tensor, pairs: torch.Tensor, params: Params,
                reps: int = 2, tcodes: torch.Tensor = None, toffsets: torch.Tensor = None):
    """pastis_autotune_sw over the given pairs (targets in codes/offsets unless tcodes/
    toffsets are given).  Sets the chosen layout on ctx and returns (layout uint8[64],
    cycles int64[4, 64]: rows 0-2 the extra stripes, row 3 the 32-bit lanes)."""
    L = _layout_sigs()
    tcodes = codes if tcodes is None else tcodes
    toffsets = offsets if toffsets is None else toffsets
    extra = np.zeros(SW_BINS, np.uint8)
    cyc = np.zeros((SW_MAX_EXTRA + 2, SW_BINS), np.int64)
    p = params.c()
    _check("pastis_autotune_sw", L.pastis_autotune_sw(ctx.h, _ptr(codes), _ptr(offsets), offsets.numel() - 1,
                                                      _ptr(tcodes), _ptr(toffsets), toffsets.numel() - 1,
                                                      _ptr(pairs), pairs.shape[0], ctypes.byref(p), reps,
                                                      extra.ctypes.data_as(ctypes.c_void_p),
                                                      cyc.ctypes.data_as(ctypes.c_void_p)))
    return extra, cyc


XD_CHOICES = (0, 1, 2, 4)


def autotune_xd(ctx: Context, codes: torch.Tensor, offsets: torch.Tensor, pairs: torch.Tensor, params: Params,
                reps: int = 2, tcodes: torch.Tensor = None, toffsets: torch.Tensor = None):
    """pastis_autotune_xd over the given pairs.  Sets the chosen x-drop layout on ctx and
    returns (per_warp, {setting: best ms}) for the settings 0, 1, 2, 4."""
    L = _layout_sigs()
    tcodes = codes if tcodes is None else tcodes
    toffsets = offsets if toffsets is None else toffsets
    pw = ctypes.c_int32()
    ms = (ctypes.c_double * 4)()
    p = params.c()
    _check("pastis_autotune_xd", L.pastis_autotune_xd(ctx.h, _ptr(codes), _ptr(offsets), offsets.numel() - 1,
                                                      _ptr(tcodes), _ptr(toffsets), toffsets.numel() - 1,
                                                      _ptr(pairs), pairs.shape[0], ctypes.byref(p), reps,
                                                      ctypes.byref(pw), ms))
    return pw.value, {c: ms[x] for x, c in enumerate(XD_CHOICES)}


def _plan_sigs():
    L = lib()
    if not getattr(L, "_plan_sigs", False):
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.pastis_align_plan_create.argtypes = [P, P, P, i32, i32, i64, i64, i32, ctypes.POINTER(c_params),
                                               ctypes.POINTER(P)]
        L.pastis_align_plan_create.restype = i32
        L.pastis_align_plan_run.argtypes = [P, P, P, i32, P, i64, P]
        L.pastis_align_plan_run.restype = i32
        L.pastis_align_plan_destroy.argtypes = [P]
        L.pastis_align_plan_destroy.restype = i32
        L.pastis_align_plan_graph_nodes.argtypes = [P]
        L.pastis_align_plan_graph_nodes.restype = i64
        L._plan_sigs = True
    return L


class AlignPlan:
    """pastis_align_plan: the alignment of a batch of queries against resident targets,
    captured once as a CUDA graph over buffers of fixed capacity and replayed per batch
    (one graph launch per run).  Runs on ctx's stream."""

    def __init__(self, ctx: Context, tcodes: torch.Tensor, toffsets: torch.Tensor, params: Params,
                 max_q: int, max_qres: int, max_pairs: int, max_len: int):
        L = _plan_sigs()
        self._targets = (tcodes, toffsets)          # the plan reads them on every run
        self.max_q, self.max_qres, self.max_pairs, self.max_len = max_q, max_qres, max_pairs, max_len
        p = params.c()
        h = ctypes.c_void_p()
        _check("pastis_align_plan_create", L.pastis_align_plan_create(
            ctx.h, _ptr(tcodes), _ptr(toffsets), toffsets.numel() - 1, max_q, max_qres, max_pairs, max_len,
            ctypes.byref(p), ctypes.byref(h)))
        self.h = h
        self.device = tcodes.device

    def fits(self, qoffsets_host: np.ndarray, n_pairs: int) -> bool:
        n_q = qoffsets_host.shape[0] - 1
        return (1 <= n_q <= self.max_q and n_pairs <= self.max_pairs and int(qoffsets_host[-1]) <= self.max_qres
                and int(np.diff(qoffsets_host).max(initial=0)) <= self.max_len)

    def run(self, qcodes: torch.Tensor, qoffsets_host: np.ndarray, pairs: torch.Tensor,
            out: torch.Tensor = None) -> torch.Tensor:
        """pastis_align_plan_run: one record (uint8 [n, 20]) per pair."""
        qo = np.ascontiguousarray(qoffsets_host, dtype=np.int64)
        n = pairs.shape[0]
        out = torch.empty((max(n, 1), REC_BYTES), dtype=torch.uint8, device=self.device) if out is None else out
        _check("pastis_align_plan_run", _plan_sigs().pastis_align_plan_run(
            self.h, _ptr(qcodes), qo.ctypes.data_as(ctypes.c_void_p), qo.shape[0] - 1, _ptr(pairs), n, _ptr(out)))
        return out[:n]

    @property
    def graph_nodes(self) -> int:
        return int(_plan_sigs().pastis_align_plan_graph_nodes(self.h))

    def close(self):
        if getattr(self, "h", None):
            _plan_sigs().pastis_align_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def filter_edges(ctx: Context, offsets: torch.Tensor, pairs: torch.Tensor, alns: torch.Tensor,
                 params: Params) -> torch.Tensor:
    """pastis_filter_edges: edges (uint8 [n, 20]) of the pairs that pass, in pair order."""
    n = pairs.shape[0]
    p = params.c()
    nout = ctypes.c_int64()
    cap = max(1, n)
    out = torch.empty((cap, REC_BYTES), dtype=torch.uint8, device=offsets.device)
    _check("pastis_filter_edges", lib().pastis_filter_edges(ctx.h, _ptr(offsets), offsets.numel() - 1, _ptr(pairs),
                                                            _ptr(alns), n, ctypes.byref(p), _ptr(out), cap,
                                                            ctypes.byref(nout)))
    return out[:nout.value]


def _variant_sigs(L):
    if not getattr(L, "_variant_sigs", False):
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.pastis_ns_edges.argtypes = [P, P, i32, P, P, i64, P, i64, ctypes.POINTER(i64)]
        L.pastis_ns_edges.restype = i32
        L.pastis_components.argtypes = [P, i32, P, i64, P]
        L.pastis_components.restype = i32
        L._variant_sigs = True
    return L


def ns_edges(ctx: Context, offsets: torch.Tensor, pairs: torch.Tensor, alns: torch.Tensor) -> torch.Tensor:
    """pastis_ns_edges: edges weighted by score / shorter length (uint8 [n, 20]), pair order."""
    L = _variant_sigs(lib())
    n = pairs.shape[0]
    nout = ctypes.c_int64()
    cap = max(1, n)
    out = torch.empty((cap, REC_BYTES), dtype=torch.uint8, device=offsets.device)
    _check("pastis_ns_edges", L.pastis_ns_edges(ctx.h, _ptr(offsets), offsets.numel() - 1, _ptr(pairs), _ptr(alns),
                                                n, _ptr(out), cap, ctypes.byref(nout)))
    return out[:nout.value]


def components(ctx: Context, n_seqs: int, edges: torch.Tensor) -> torch.Tensor:
    """pastis_components: int32 label per sequence = smallest sequence of its component."""
    L = _variant_sigs(lib())
    labels = torch.empty(max(1, n_seqs), dtype=torch.int32, device=edges.device)
    _check("pastis_components", L.pastis_components(ctx.h, n_seqs, _ptr(edges), edges.shape[0], _ptr(labels)))
    return labels[:n_seqs]


FILTER_STATIC_MAX_PAIRS = 4194304      # PASTIS_FILTER_STATIC_MAX_PAIRS


def filter_edges_static(stream: torch.cuda.Stream, offsets: torch.Tensor, pairs: torch.Tensor, alns: torch.Tensor,
                        params: Params, out: torch.Tensor) -> int:
    """pastis_filter_edges_static: the filter into the caller's `out` (uint8 [cap, 20])
    with no allocation inside the call; returns the number of edges written.  Calls on
    one device must not overlap in time (they share one scratch array)."""
    L = lib()
    if not getattr(L, "_static_sigs", False):
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.pastis_filter_edges_static.argtypes = [P, P, i32, P, P, i64, ctypes.POINTER(c_params), P, i64,
                                                 ctypes.POINTER(i64)]
        L.pastis_filter_edges_static.restype = i32
        L._static_sigs = True
    n = pairs.shape[0]
    if n > FILTER_STATIC_MAX_PAIRS:
        raise PastisError("pastis_filter_edges_static", 7, f"n_pairs {n} exceeds {FILTER_STATIC_MAX_PAIRS}")
    p = params.c()
    nout = ctypes.c_int64()
    _check("pastis_filter_edges_static", L.pastis_filter_edges_static(
        ctypes.c_void_p(stream.cuda_stream), _ptr(offsets), offsets.numel() - 1, _ptr(pairs), _ptr(alns), n,
        ctypes.byref(p), _ptr(out), out.shape[0], ctypes.byref(nout)))
    return nout.value


PROBE_KINDS = {"viaddmax_s16x2": 0, "vimax3_s16x2_relu": 1, "vadd2": 2, "prmt": 3, "imad": 4, "imax": 5,
               "lop3": 6, "iadd": 7, "sw_mix": 8, "max3_add2": 9}


def probe_int_throughput(ctx: Context, kind: str, blocks_per_sm: int = 4, iters: int = 20000) -> float:
    """pastis_probe_int_throughput: measured warp-instructions per SM clock of one integer
    instruction kind (or the pass-1 recurrence mix) over every SM."""
    L = lib()
    if not getattr(L, "_probe_sigs", False):
        L.pastis_probe_int_throughput.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                  ctypes.POINTER(ctypes.c_double)]
        L.pastis_probe_int_throughput.restype = ctypes.c_int32
        L._probe_sigs = True
    out = ctypes.c_double()
    _check("pastis_probe_int_throughput", L.pastis_probe_int_throughput(ctx.h, PROBE_KINDS[kind], blocks_per_sm,
                                                                        iters, ctypes.byref(out)))
    return out.value


def to_records(t: torch.Tensor, dtype: np.dtype) -> np.ndarray:
    """Device record bytes -> numpy structured array (host copy)."""
    a = t.detach().to("cpu").contiguous().numpy()
    return a.reshape(-1).view(dtype).copy() if a.size else np.zeros(0, dtype)


def run(ctx: Context, ascii_dev: torch.Tensor, offsets_dev: torch.Tensor, params: Params,
        cells: torch.Tensor = None, rows=None) -> dict:
    """The whole path a1..a10 on the device; rows=(i0, i1) limits the candidates to the
    queries i0 <= i < i1 (against every j > i)."""
    codes = encode(ctx, ascii_dev)
    A = build_kmers(ctx, codes, offsets_dev, params.k)
    cands = overlap_spgemm(ctx, A, params, rows=rows)
    alns = align_pairs(ctx, codes, offsets_dev, cands, params, cells)
    edges = filter_edges(ctx, offsets_dev, cands, alns, params)
    return dict(codes=codes, A=A, cands=cands, alns=alns, edges=edges)
