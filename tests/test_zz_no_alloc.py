"""pastis_filter_edges_static (the filter with its scratch in a fixed device array, no
allocation inside the call) against pastis_filter_edges on the same inputs: identical
edges on two calls in a row, for real candidates and at the maximum size, plus its
size limit, capacity and bad-index errors.  Collected last on purpose: it must pass
both alone in a fresh process and after every other test."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
MAT = synth.blosum62()


@pytest.fixture(scope="module")
def env():
    from paper_2009_14467_gb300 import pastis as P
    ctx = P.Context(0)
    yield P, ctx
    ctx.close()


def _static_raw(P, stream, offsets, pairs, alns, n, params, out, cap):
    """The C call itself, with no size check on the Python side."""
    L = P.lib()
    Pp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.pastis_filter_edges_static.argtypes = [Pp, Pp, i32, Pp, Pp, i64, ctypes.POINTER(P.c_params), Pp, i64,
                                             ctypes.POINTER(i64)]
    L.pastis_filter_edges_static.restype = i32
    nout = ctypes.c_int64()
    p = params.c()
    st = L.pastis_filter_edges_static(ctypes.c_void_p(stream.cuda_stream), P._ptr(offsets), offsets.numel() - 1,
                                      P._ptr(pairs), P._ptr(alns), n, ctypes.byref(p), P._ptr(out), cap,
                                      ctypes.byref(nout))
    return st, nout.value


def _both(P, ctx, offsets, pairs, alns, params):
    ref = P.to_records(P.filter_edges(ctx, offsets, pairs, alns, params), P.EDGE_DTYPE)
    stream = torch.cuda.current_stream()
    got = []
    for _ in range(2):                                   # two calls in a row
        out = torch.full((max(pairs.shape[0], 1), P.REC_BYTES), 0xAB, dtype=torch.uint8, device="cuda")
        n = P.filter_edges_static(stream, offsets, pairs, alns, params, out)
        got.append(P.to_records(out[:n], P.EDGE_DTYPE))
    return ref, got


def test_static_filter_equals_filter_on_candidates(env):
    P, ctx = env
    ps = synth.families_1k()
    params = P.Params(matrix=MAT)
    a = torch.from_numpy(ps.ascii).cuda()
    o = torch.from_numpy(ps.offsets).cuda()
    codes = P.encode(ctx, a)
    A = P.build_kmers(ctx, codes, o, 6)
    cands = P.overlap_spgemm(ctx, A, params)
    alns = P.align_pairs(ctx, codes, o, cands, params)
    ref, got = _both(P, ctx, o, cands, alns, params)
    assert cands.shape[0] > 3 * 1024 and len(ref) > 0       # several tiles and a ragged tail
    for g in got:
        assert g.tobytes() == ref.tobytes()



def test_static_filter_allocates_nothing_and_matches_oracle(env):
    """The call's defining property: with the caller's buffers in place, a call leaves
    the device's free memory unchanged.  And its edges equal the oracle's filter applied
    to the same alignments."""
    from oracle import oracle as O
    P, ctx = env
    ps = synth.families_1k()
    params = P.Params(matrix=MAT)
    a = torch.from_numpy(ps.ascii).cuda()
    o = torch.from_numpy(ps.offsets).cuda()
    codes = P.encode(ctx, a)
    A = P.build_kmers(ctx, codes, o, 6)
    cands = P.overlap_spgemm(ctx, A, params)
    alns = P.align_pairs(ctx, codes, o, cands, params)
    stream = torch.cuda.current_stream()
    out = torch.zeros((cands.shape[0], P.REC_BYTES), dtype=torch.uint8, device="cuda")
    P.filter_edges_static(stream, o, cands, alns, params, out)     # first call: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n = P.filter_edges_static(stream, o, cands, alns, params, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    want = O.filter_edges(ps.offsets, P.to_records(cands, P.CAND_DTYPE), P.to_records(alns, P.ALN_DTYPE))
    assert len(want) > 0
    assert P.to_records(out[:n], P.EDGE_DTYPE).tobytes() == want.tobytes()


def _random_records(P, n, n_seqs, seed):
    rng = np.random.default_rng(seed)
    lens = rng.integers(50, 1001, size=n_seqs)
    offs = np.zeros(n_seqs + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    pairs = np.zeros(n, P.CAND_DTYPE)
    pairs["i"] = rng.integers(0, n_seqs, size=n)
    pairs["j"] = rng.integers(0, n_seqs, size=n)
    alns = np.zeros(n, P.ALN_DTYPE)
    li, lj = lens[pairs["i"]], lens[pairs["j"]]
    qb = (rng.random(n) * 0.4 * li).astype(np.int64)
    tb = (rng.random(n) * 0.4 * lj).astype(np.int64)
    alns["qb"], alns["tb"] = qb, tb
    alns["qe"] = qb + ((li - qb) * rng.random(n)).astype(np.int64)
    alns["te"] = tb + ((lj - tb) * rng.random(n)).astype(np.int64)
    cols = rng.integers(0, 1200, size=n)
    alns["cols"] = cols
    alns["ident"] = (cols * rng.random(n)).astype(np.int64)
    alns["score"] = rng.integers(0, 3000, size=n)
    dev = lambda x: torch.from_numpy(x.view(np.uint8).reshape(n, 20)).cuda()
    return torch.from_numpy(offs).cuda(), dev(pairs), dev(alns)


def test_static_filter_at_maximum_size(env):
    P, ctx = env
    n = P.FILTER_STATIC_MAX_PAIRS
    o, pairs, alns = _random_records(P, n, 5000, 3)
    ref, got = _both(P, ctx, o, pairs, alns, P.Params(matrix=MAT))
    assert 0 < len(ref) < n
    for g in got:
        assert g.tobytes() == ref.tobytes()


def test_static_filter_errors(env):
    P, ctx = env
    params = P.Params(matrix=MAT)
    stream = torch.cuda.current_stream()
    L = P.lib()
    # one pair above the limit: rejected before any work (buffers valid for every pair anyway)
    n = P.FILTER_STATIC_MAX_PAIRS + 1
    o = torch.tensor([0, 100], dtype=torch.int64, device="cuda")
    pairs = torch.zeros((n, 20), dtype=torch.uint8, device="cuda")
    alns = torch.zeros((n, 20), dtype=torch.uint8, device="cuda")
    out = torch.zeros((n, 20), dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PastisError):
        P.filter_edges_static(stream, o, pairs, alns, params, out)
    st, _ = _static_raw(P, stream, o, pairs, alns, n, params, out, n)
    assert st == 7                                       # PASTIS_ERR_UNSUPPORTED
    # too small a capacity: the needed count comes back and nothing is written
    o2, p2, a2 = _random_records(P, 5000, 300, 4)
    ref = P.to_records(P.filter_edges(ctx, o2, p2, a2, params), P.EDGE_DTYPE)
    assert len(ref) > 1
    out2 = torch.full((len(ref) - 1, 20), 0xAB, dtype=torch.uint8, device="cuda")
    st, need = _static_raw(P, stream, o2, p2, a2, 5000, params, out2, len(ref) - 1)
    assert st == P.ERR_CAPACITY and need == len(ref)
    assert bool((out2 == 0xAB).all())
    # a pair index outside [0, n_seqs): the kernel's bounds check reports it
    bad = P.to_records(p2, P.CAND_DTYPE)
    bad["j"][17] = 300
    pb = torch.from_numpy(bad.view(np.uint8).reshape(-1, 20)).cuda()
    st, _ = _static_raw(P, stream, o2, pb, a2, 5000, params, out2, len(ref) - 1)
    assert st == 1                                       # PASTIS_ERR_INVALID_ARG
    # a good call right after the errors still gives the filter's edges
    out3 = torch.zeros((5000, 20), dtype=torch.uint8, device="cuda")
    k = P.filter_edges_static(stream, o2, p2, a2, params, out3)
    assert P.to_records(out3[:k], P.EDGE_DTYPE).tobytes() == ref.tobytes()
