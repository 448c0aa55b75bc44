"""What the trained prefilter gains over the path without it.

The network is trained by the library's own kernels on pass/fail labels that the exact
path produces (the filter verdict of Sec. IV-F on every candidate of one row block of a
20,000-protein planted-family set with 25 substitute k-mers), its threshold is
calibrated for recall on a second block, and it is judged on a held-out third block
against the exact alignment of every candidate there.  The paper's own way to trade a
little recall for fewer alignments is the common-k-mer threshold (Sec. VI: dropping
pairs that share few k-mers removes most alignments for a few percent of recall); the
network is compared with it at the recall that threshold reaches."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
MAT = synth.blosum62()


def _row_blocks(n, parts):
    """Query-row ranges of equal all-vs-all work (row i pairs with the n-1-i rows after it)."""
    work = np.arange(n - 1, -1, -1, dtype=np.float64)
    cum = np.concatenate([[0.0], np.cumsum(work)])
    cuts = [int(np.searchsorted(cum, cum[-1] * k / parts)) for k in range(1, parts)]
    b = [0] + cuts + [n]
    return [(b[k], b[k + 1]) for k in range(parts)]


@pytest.fixture(scope="module")
def env():
    import paper_2009_14467_gb300 as P
    from paper_2009_14467_gb300 import prefilter as F
    ctx = P.Context(0)
    ps = synth.zipf_100k(n=20000)
    a = torch.from_numpy(ps.ascii).cuda()
    o = torch.from_numpy(ps.offsets).cuda()
    params = P.Params(matrix=MAT, m_subs=25, mode=P.SW_FILTERED)
    codes = P.encode(ctx, a)
    A = P.build_kmers(ctx, codes, o, 6)
    yield P, F, ctx, ps, codes, o, A, params
    ctx.close()


def _exact(P, ctx, codes, o, A, params, rows):
    cands = P.overlap_spgemm(ctx, A, params, rows=rows)
    alns = P.align_pairs(ctx, codes, o, cands, params)
    edges = P.filter_edges(ctx, o, cands, alns, params)
    return cands, alns, edges


def _edge_keys(P, edges):
    e = P.to_records(edges, P.EDGE_DTYPE)
    return e, set(zip(e["i"].tolist(), e["j"].tolist()))


def test_trained_prefilter_gain(env):
    P, F, ctx, ps, codes, o, A, params = env
    blocks = _row_blocks(ps.n, 4)
    # train on the exact path's verdicts of block 0
    c0, a0, _ = _exact(P, ctx, codes, o, A, params, blocks[0])
    y0 = F.labels_from(a0)
    assert 0 < float(y0.sum()) < y0.numel()
    net = F.MLP(seed=11)
    hist = F.train(ctx, net, F.features(ctx, codes, o, c0, params), y0, epochs=3, batch=65536, lr=2e-3, seed=13)
    assert hist[-1] < hist[0]
    del c0, a0, y0
    # calibrate on block 1
    c1, a1, _ = _exact(P, ctx, codes, o, A, params, blocks[1])
    thr = F.threshold_for_recall(F.forward(ctx, net, F.features(ctx, codes, o, c1, params)), F.labels_from(a1), 0.998)
    del c1, a1
    # held-out block 2: every candidate aligned exactly, against the prefiltered path
    c2, a2, e2 = _exact(P, ctx, codes, o, A, params, blocks[2])
    z2 = F.forward(ctx, net, F.features(ctx, codes, o, c2, params))
    kept = F.select(ctx, c2, z2, thr)
    ak = P.align_pairs(ctx, codes, o, kept, params)
    ek = P.filter_edges(ctx, o, kept, ak, params)
    exact, exact_keys = _edge_keys(P, e2)
    got, got_keys = _edge_keys(P, ek)
    assert len(exact) > 1000
    # every prefiltered edge is an exact edge, record for record
    assert got_keys <= exact_keys
    pos = {k: x for x, k in enumerate(zip(exact["i"].tolist(), exact["j"].tolist()))}
    idx = np.array([pos[k] for k in zip(got["i"].tolist(), got["j"].tolist())], np.int64)
    assert got.tobytes() == exact[idx].tobytes()
    recall = len(got) / len(exact)
    reduction = 1.0 - kept.shape[0] / c2.shape[0]
    assert recall >= 0.995, recall
    assert reduction >= 0.5, reduction              # at least half of the alignments skipped
    # against the common-k-mer threshold at the recall it reaches
    y2 = F.labels_from(a2)
    for min_shared in (2, 4):
        pk = P.Params(matrix=MAT, m_subs=25, mode=P.SW_FILTERED, min_shared=min_shared)
        ck, _, eck = _exact(P, ctx, codes, o, A, pk, blocks[2])
        r_ck = eck.shape[0] / len(exact)
        frac_ck = ck.shape[0] / c2.shape[0]
        thr_ck = F.threshold_for_recall(z2, y2, r_ck)
        frac_net = float((z2 >= thr_ck).float().mean())
        assert frac_net <= frac_ck, (min_shared, r_ck, frac_ck, frac_net)
