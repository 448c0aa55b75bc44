"""GPU parity of the graph variants (Sec. VI-B) with the oracle: the score-only
alignment mode (the NS weight needs no traceback), NS edges, and connected components
of the edge graph; all bit-exact."""
import numpy as np
import pytest
import torch

import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu
MAT = synth.blosum62()


@pytest.fixture(scope="module")
def env():
    from paper_2009_14467_gb300 import pastis as P
    ctx = P.Context(0)
    yield P, ctx
    ctx.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def recs(a):
    return dev(a.view(np.uint8).reshape(-1, 20))


def _pairs(n):
    i, j = np.triu_indices(n, 1)
    c = np.zeros(i.size, O.CAND_DTYPE)
    c["i"], c["j"], c["count"] = i, j, 1
    return c


def _cands(ps):
    codes = O.encode(ps.ascii)
    rp, code, pos = O.kmers(codes, ps.offsets, 6)
    return codes, O.candidates(rp, code, pos, 6, 0, MAT, 1)


@pytest.mark.parametrize("which", ["families", "long"])
def test_score_mode_and_ns_edges(env, which):
    P, ctx = env
    if which == "families":
        ps = synth.families_1k()
        codes, c = _cands(ps)
    else:
        # shorter length >= 2909 makes 11 * length reach the packed pass's score limit,
        # so these pairs take the int32 whole-matrix path
        ps = synth.planted_families([3], 1, (2950, 3100), seed=8)
        codes = O.encode(ps.ascii)
        c = _pairs(ps.n)
    params = P.Params(matrix=MAT, mode=P.SW_SCORE)
    got = P.to_records(P.align_pairs(ctx, dev(codes), dev(ps.offsets), recs(c), params), P.ALN_DTYPE)
    want, _ = O.align_pairs(codes, ps.offsets, c, MAT, mode=O.SW_SCORE)
    assert got.tobytes() == want.tobytes()
    e = P.to_records(P.ns_edges(ctx, dev(ps.offsets), recs(c), recs(want)), P.EDGE_DTYPE)
    assert e.tobytes() == O.ns_edges(ps.offsets, c, want).tobytes()
    assert (e["weight"] > 0).all()


def _edges(a, b):
    e = np.zeros(len(a), O.EDGE_DTYPE)
    e["i"], e["j"] = a, b
    return e


def test_components_of_the_similarity_graph(env):
    P, ctx = env
    ps = synth.families_1k()
    codes, c = _cands(ps)
    alns, _ = O.align_pairs(codes, ps.offsets, c, MAT)
    edges = O.filter_edges(ps.offsets, c, alns)
    lab = P.components(ctx, ps.n, recs(edges)).cpu().numpy()
    ref = O.components(ps.n, edges)
    assert (lab == ref).all()
    p, r = O.weighted_precision_recall(lab, ps.family)
    assert 0.9 < p <= 1.0 and 0.5 < r <= 1.0


@pytest.mark.parametrize("n,m", [(1, 0), (50, 0), (5000, 20000), (20000, 19000), (3000, 60000)])
def test_components_random_graphs(env, n, m):
    P, ctx = env
    rng = np.random.default_rng(n + m)
    a = rng.integers(0, n, size=m)
    b = rng.integers(0, n, size=m)
    if m:
        b[:m // 10] = a[:m // 10]                    # self loops and repeats
    e = _edges(a, b)
    lab = P.components(ctx, n, recs(e) if m else torch.zeros((0, 20), dtype=torch.uint8, device="cuda"))
    assert (lab.cpu().numpy() == O.components(n, e)).all()


def test_components_reject_bad_endpoint(env):
    P, ctx = env
    e = _edges([0, 1], [1, 7])
    with pytest.raises(P.PastisError):
        P.components(ctx, 5, recs(e))
