"""Serving loop: query batches against a device-resident database index, with
continuous batching.

The database (residue codes, offsets and its sequence x k-mer matrix in CSR + CSC) is
built once and stays on the device.  Requests (a batch of 1..4096 query proteins each)
enter a queue; `slots` worker threads, each with its own CUDA stream and library
context, take the next request as soon as they are free and the device has room for
it (admission by free device memory), so requests that arrive while others run are
admitted as slots and memory free up, and their kernels overlap on the GPU.  Each
request runs the hot path in serving form: encode -> query k-mer matrix -> query x
database candidates -> (optional learned prefilter) -> alignment -> filter, and
returns the edges (query index, database index, ident, cols, score, ANI).  With
`chunk_queries` > 0 a larger request runs as chunks of consecutive queries that the
slots take like requests of their own, in rounds across requests, its edges joined in
query order.  Each
worker's alignment of a request within the plan's capacities is one replay of a CUDA
graph captured at the worker's start (pastis_align_plan); larger requests take the
direct call, with the same records.  Every numeric step is a library kernel; this
module only schedules.
"""
import concurrent.futures
import ctypes
import itertools
import queue
import threading
import time

import numpy as np
import torch

from . import pastis as P


ADMIT_WAIT_S = 30.0


def admissible(free: int, in_flight: int, reserve: int, need: int, waited: float) -> bool:
    """Admission by device memory: a request starts when the free memory, less what the
    requests already admitted may still take and a reserve, covers its estimate; always
    when nothing else is in flight (it cannot wait for memory nobody will free), and
    after waiting ADMIT_WAIT_S (so that an estimate set too high cannot stall it)."""
    return free - in_flight - reserve >= need or in_flight == 0 or waited > ADMIT_WAIT_S


def query_chunks(n: int, chunk: int):
    """Query ranges [c0, c1) of at most `chunk` queries covering [0, n), in order."""
    if chunk <= 0 or n <= chunk:
        return [(0, n)]
    k = -(-n // chunk)
    return [(n * x // k, n * (x + 1) // k) for x in range(k)]


class Request:
    def __init__(self, ascii_host: np.ndarray, offsets_host: np.ndarray, rid: int):
        self.ascii = ascii_host
        self.offsets = offsets_host
        self.rid = rid
        self.n = int(offsets_host.shape[0] - 1)
        self.t_submit = time.perf_counter()
        self.t_start = None
        self.t_done = None
        self.future = concurrent.futures.Future()
        self.parent = None                  # a chunk: (request, chunk index, first query)
        self.parts = None                   # a split request: its chunks' edges
        self.left = 0
        self.lock = threading.Lock()


def _kmat_c(A):
    return A.c()


class Server:
    """Query batches against a resident database."""

    def __init__(self, db_ascii: np.ndarray, db_offsets: np.ndarray, params: P.Params, device: int = 0,
                 slots: int = 4, reserve_bytes: int = 8 << 30, prefilter=None, graphs: bool = True,
                 graph_pairs: int = 1 << 20, graph_queries: int = 4096, graph_residues: int = 4 << 20,
                 chunk_queries: int = 0):
        if params.m_subs != 0:
            raise ValueError("the serving form takes exact k-mers (m_subs = 0)")
        self.params = params
        self.prefilter = prefilter          # (prefilter.MLP, threshold) or None
        self.device = torch.device("cuda", device)
        self.reserve = reserve_bytes
        torch.cuda.set_device(self.device)
        build_stream = torch.cuda.Stream(self.device)
        with torch.cuda.stream(build_stream):
            ctx = P.Context(device, build_stream)
            a = torch.from_numpy(np.ascontiguousarray(db_ascii)).to(self.device)
            self.db_offsets = torch.from_numpy(np.ascontiguousarray(db_offsets)).to(self.device)
            self.db_codes = P.encode(ctx, a)
            self.DB = P.build_kmers(ctx, self.db_codes, self.db_offsets, params.k)
            build_stream.synchronize()
            ctx.close()
        self.n_db = int(db_offsets.shape[0] - 1)
        # alignment plans (CUDA graphs), one per worker context, for requests within
        # their capacities; longer queries or more pairs take the direct call
        self.graphs = graphs
        self.graph_caps = (graph_queries, graph_residues, graph_pairs,
                           max(2000, int(np.diff(db_offsets).max(initial=0))))
        self.graph_runs = 0
        # optional: a request of more than chunk_queries queries runs as chunks that the
        # slots take independently, so small requests need not wait behind a large one
        # and a large one spreads over the slots; the chunks' edges are joined in query
        # order (the same edges).  0 (the default): whole requests, first come first served
        self.chunk_queries = chunk_queries
        # the slots take work in rounds: every request's first chunk before any request's
        # second (arrival order within a round), so a large request does not hold back the
        # requests that arrive after it
        self.q = queue.PriorityQueue()
        self.seq = itertools.count()
        self.mem_lock = threading.Lock()
        self.in_flight_bytes = 0
        self.stop = False
        self.done = []
        self.workers = [threading.Thread(target=self._worker, args=(s,), daemon=True) for s in range(slots)]
        for w in self.workers:
            w.start()

    # -- public --------------------------------------------------------------------
    def submit(self, ascii_host: np.ndarray, offsets_host: np.ndarray, rid: int = 0) -> Request:
        r = Request(ascii_host, offsets_host, rid)
        ranges = query_chunks(r.n, self.chunk_queries)
        if len(ranges) == 1:
            self.q.put((0, next(self.seq), r))
            return r
        r.parts = [None] * len(ranges)
        r.left = len(ranges)
        for x, (c0, c1) in enumerate(ranges):
            o0, o1 = int(offsets_host[c0]), int(offsets_host[c1])
            c = Request(ascii_host[o0:o1], np.ascontiguousarray(offsets_host[c0:c1 + 1] - o0), rid)
            c.t_submit = r.t_submit
            c.parent = (r, x, c0)
            self.q.put((x, next(self.seq), c))
        return r

    def _finish(self, r: Request, res=None, exc=None):
        """Completes a request, or a chunk and, with its last chunk, its request."""
        r.t_done = time.perf_counter()
        if r.parent is None:
            if exc is not None:
                r.future.set_exception(exc)
            else:
                self.done.append(r)
                r.future.set_result(res)
            return
        top, x, c0 = r.parent
        with top.lock:
            if exc is not None:
                top.parts[x] = exc
            else:
                res = res.copy()
                res["i"] += c0
                top.parts[x] = res
            top.left -= 1
            last = top.left == 0
        if last:
            top.t_done = time.perf_counter()
            bad = [p for p in top.parts if isinstance(p, BaseException)]
            if bad:
                top.future.set_exception(bad[0])
            else:
                self.done.append(top)
                top.future.set_result(np.concatenate(top.parts))

    def close(self):
        self.stop = True
        for _ in self.workers:
            self.q.put((float("inf"), next(self.seq), None))
        for w in self.workers:
            w.join(timeout=60)

    def latency_stats(self):
        lat = np.array([r.t_done - r.t_submit for r in self.done])
        nq = sum(r.n for r in self.done)
        if lat.size == 0:
            return {}
        span = max(r.t_done for r in self.done) - min(r.t_submit for r in self.done)
        return {"requests": int(lat.size), "queries": int(nq), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "queries_per_s": nq / span if span > 0 else 0.0}

    # -- the work of one request ------------------------------------------------------
    def estimate_bytes(self, r: Request) -> int:
        residues = int(r.offsets[-1])
        # query A and its sort buffers, candidates (records, alignments), alignment scratch
        return residues * 48 + r.n * 4096 * 60 + (64 << 20)

    def process(self, ctx: P.Context, r: Request) -> np.ndarray:
        dev = self.device
        a = torch.from_numpy(np.ascontiguousarray(r.ascii)).to(dev, non_blocking=True)
        o = torch.from_numpy(np.ascontiguousarray(r.offsets)).to(dev, non_blocking=True)
        codes = P.encode(ctx, a)
        Q = P.build_kmers(ctx, codes, o, self.params.k)
        cands = query_overlap(ctx, Q, self.DB, self.params)
        if self.prefilter is not None and cands.shape[0] > 0:
            from . import prefilter as F
            net, thr = self.prefilter
            z = F.forward(ctx, net, F.features_qt(ctx, codes, o, self.db_codes, self.db_offsets, cands, self.params))
            cands = F.select(ctx, cands, z, thr)
        plan = self._plan(ctx) if self.graphs else None
        if plan is not None and plan.fits(r.offsets, cands.shape[0]):
            alns = plan.run(codes, r.offsets, cands)
            self.graph_runs += 1
        else:
            alns = align_pairs_qt(ctx, codes, o, self.db_codes, self.db_offsets, cands, self.params)
        edges = filter_edges_qt(ctx, o, self.db_offsets, cands, alns, self.params)
        return P.to_records(edges, P.EDGE_DTYPE)

    def _plan(self, ctx: P.Context):
        """The context's plan for this server (made on first use, kept on the context)."""
        plan = getattr(ctx, "_serve_plan", None)
        if plan is None or plan[0] is not self:
            q, res, pairs, ln = self.graph_caps
            plan = (self, P.AlignPlan(ctx, self.db_codes, self.db_offsets, self.params, q, res, pairs, ln))
            ctx._serve_plan = plan
        return plan[1]

    def drop_plan(self, ctx: P.Context):
        """Frees the context's plan (before the context closes)."""
        plan = getattr(ctx, "_serve_plan", None)
        if plan is not None:
            plan[1].close()
            ctx._serve_plan = None

    def _worker(self, slot: int):
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(self.device)
        with torch.cuda.stream(stream):
            ctx = P.Context(self.device.index or 0, stream)
            if self.graphs:
                self._plan(ctx)             # captured before the first request
            while True:
                r = self.q.get()[2]
                if r is None:
                    break
                need = self.estimate_bytes(r)
                waited = 0.0
                while True:               # admission by free device memory (bounded wait)
                    with self.mem_lock:
                        free, _ = torch.cuda.mem_get_info(self.device)
                        if admissible(free, self.in_flight_bytes, self.reserve, need, waited):
                            self.in_flight_bytes += need
                            break
                    time.sleep(0.002)
                    waited += 0.002
                r.t_start = time.perf_counter()
                try:
                    res = self.process(ctx, r)
                    stream.synchronize()
                    self._finish(r, res=res)
                except Exception as exc:       # the request fails, the server keeps going
                    self._finish(r, exc=exc)
                finally:
                    with self.mem_lock:
                        self.in_flight_bytes -= need
            self.drop_plan(ctx)
            ctx.close()


# ---- bindings of the serving-form entry points ---------------------------------------
def _sigs():
    L = P.lib()
    if not getattr(L, "_serve_sigs", False):
        Pp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.pastis_query_overlap.argtypes = [Pp, ctypes.POINTER(P.c_kmat), ctypes.POINTER(P.c_kmat),
                                           ctypes.POINTER(P.c_params), Pp, i64, ctypes.POINTER(i64)]
        L.pastis_query_overlap.restype = i32
        L.pastis_align_pairs_qt.argtypes = [Pp, Pp, Pp, i32, Pp, Pp, i32, Pp, i64, ctypes.POINTER(P.c_params), Pp, Pp]
        L.pastis_align_pairs_qt.restype = i32
        L.pastis_filter_edges_qt.argtypes = [Pp, Pp, i32, Pp, i32, Pp, Pp, i64, ctypes.POINTER(P.c_params), Pp, i64,
                                             ctypes.POINTER(i64)]
        L.pastis_filter_edges_qt.restype = i32
        L._serve_sigs = True
    return L


def query_overlap(ctx, Q, DB, params) -> torch.Tensor:
    L = _sigs()
    p, qm, dm = params.c(), Q.c(), DB.c()
    nout = ctypes.c_int64()
    st = L.pastis_query_overlap(ctx.h, ctypes.byref(qm), ctypes.byref(dm), ctypes.byref(p), None, 0,
                                ctypes.byref(nout))
    if st not in (0, P.ERR_CAPACITY):
        P._check("pastis_query_overlap", st)
    out = torch.empty((max(nout.value, 1), P.REC_BYTES), dtype=torch.uint8, device=Q.row_ptr.device)
    if nout.value > 0:
        P._check("pastis_query_overlap", L.pastis_query_overlap(ctx.h, ctypes.byref(qm), ctypes.byref(dm),
                                                                ctypes.byref(p), P._ptr(out), nout.value,
                                                                ctypes.byref(nout)))
    return out[:nout.value]


def align_pairs_qt(ctx, qcodes, qoff, tcodes, toff, pairs, params, cells=None) -> torch.Tensor:
    L = _sigs()
    n = pairs.shape[0]
    out = torch.empty((max(n, 1), P.REC_BYTES), dtype=torch.uint8, device=qcodes.device)
    p = params.c()
    P._check("pastis_align_pairs_qt", L.pastis_align_pairs_qt(
        ctx.h, P._ptr(qcodes), P._ptr(qoff), qoff.numel() - 1, P._ptr(tcodes), P._ptr(toff), toff.numel() - 1,
        P._ptr(pairs), n, ctypes.byref(p), P._ptr(out), P._ptr(cells)))
    return out[:n]


def filter_edges_qt(ctx, qoff, toff, pairs, alns, params) -> torch.Tensor:
    L = _sigs()
    n = pairs.shape[0]
    p = params.c()
    nout = ctypes.c_int64()
    out = torch.empty((max(n, 1), P.REC_BYTES), dtype=torch.uint8, device=qoff.device)
    P._check("pastis_filter_edges_qt", L.pastis_filter_edges_qt(
        ctx.h, P._ptr(qoff), qoff.numel() - 1, P._ptr(toff), toff.numel() - 1, P._ptr(pairs), P._ptr(alns), n,
        ctypes.byref(p), P._ptr(out), max(n, 1), ctypes.byref(nout)))
    return out[:nout.value]
