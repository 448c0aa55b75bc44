"""Serving loop on the GPU: query batches against a resident database.  Each request's
edges equal the oracle's (queries placed first in a combined set, so the query is the
row of every alignment), and equal whether the request runs alone or in a mix of
concurrent requests."""
import numpy as np
import pytest
import torch

import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu
MAT = synth.blosum62()


def _requests():
    db = synth.families_1k()
    rng = np.random.default_rng(21)
    other = synth.families_1k(seed=9)
    reqs = []
    for r, size in enumerate([1, 3, 17, 64, 5, 128, 2, 40]):
        ids = rng.choice(db.n, size=size, replace=False)
        part = db.subset(ids) if r % 2 == 0 else other.subset(rng.choice(other.n, size=size, replace=False))
        reqs.append(part)
    return db, reqs


@pytest.fixture(scope="module")
def server():
    import paper_2009_14467_gb300 as P
    from paper_2009_14467_gb300 import serve as S
    db, reqs = _requests()
    srv = S.Server(db.ascii, db.offsets, P.Params(matrix=MAT), slots=4, reserve_bytes=1 << 30)
    yield P, srv, db, reqs
    srv.close()


def test_serving_matches_oracle_alone_and_in_the_mix(server):
    P, srv, db, reqs = server
    alone = []
    for r, q in enumerate(reqs):
        h = srv.submit(q.ascii, q.offsets, r)
        alone.append(h.future.result(timeout=120))
    # oracle on [queries, database]: the pair (query i, database j) is (i, nq + j), the
    # query being the row of its alignment; only those cross pairs are aligned
    for q, got in zip(reqs[:5], alone[:5]):
        both = synth.from_strings([q.seq(i) for i in range(q.n)] + [db.seq(j) for j in range(db.n)])
        codes = O.encode(both.ascii)
        rp, code, pos = O.kmers(codes, both.offsets, 6)
        c = O.candidates(rp, code, pos, 6, 0, MAT, 1)
        c = c[(c["i"] < q.n) & (c["j"] >= q.n)]
        alns, _ = O.align_pairs(codes, both.offsets, c, MAT)
        ref = O.filter_edges(both.offsets, c, alns)
        ref["j"] -= q.n
        assert got.tobytes() == ref.tobytes()
    # all at once: requests arrive while others run
    handles = [srv.submit(q.ascii, q.offsets, 100 + r) for r, q in enumerate(reqs)]
    mixed = [h.future.result(timeout=300) for h in handles]
    for a, m in zip(alone, mixed):
        assert a.tobytes() == m.tobytes()
    st = srv.latency_stats()
    assert st["requests"] >= 2 * len(reqs) and st["p99_s"] >= st["p50_s"] > 0


def test_features_qt_equal_features_of_the_joined_set(server):
    P, srv, db, reqs = server
    from paper_2009_14467_gb300 import pastis as PP, prefilter as F
    q = reqs[3]
    ctx = PP.Context(0)
    codes_q = PP.encode(ctx, torch.from_numpy(q.ascii).cuda())
    oq = torch.from_numpy(q.offsets).cuda()
    Q = PP.build_kmers(ctx, codes_q, oq, 6)
    from paper_2009_14467_gb300 import serve as S
    cands = S.query_overlap(ctx, Q, srv.DB, srv.params)
    x_qt = F.features_qt(ctx, codes_q, oq, srv.db_codes, srv.db_offsets, cands, srv.params)
    both = synth.from_strings([q.seq(i) for i in range(q.n)] + [db.seq(j) for j in range(db.n)])
    codes_b = PP.encode(ctx, torch.from_numpy(both.ascii).cuda())
    rec = PP.to_records(cands, PP.CAND_DTYPE)
    rec["j"] += q.n
    x_b = F.features(ctx, codes_b, torch.from_numpy(both.offsets).cuda(),
                     torch.from_numpy(rec.view(np.uint8).reshape(-1, 20)).cuda(), srv.params)
    assert cands.shape[0] > 0 and torch.equal(x_qt.view(torch.int16), x_b.view(torch.int16))
    ctx.close()


def test_serving_with_prefilter_alone_equals_mixed(server):
    P, srv, db, reqs = server
    from paper_2009_14467_gb300 import pastis as PP, prefilter as F, serve as S
    net = F.MLP(seed=3)
    # threshold: the median logit over one request's candidates (keeps about half)
    ctx = PP.Context(0)
    q = reqs[5]
    codes = PP.encode(ctx, torch.from_numpy(q.ascii).cuda())
    o = torch.from_numpy(q.offsets).cuda()
    cands = S.query_overlap(ctx, PP.build_kmers(ctx, codes, o, 6), srv.DB, srv.params)
    z = F.forward(ctx, net, F.features_qt(ctx, codes, o, srv.db_codes, srv.db_offsets, cands, srv.params))
    thr = float(z.median().item())
    ctx.close()
    pf = S.Server(db.ascii, db.offsets, srv.params, slots=3, reserve_bytes=1 << 30, prefilter=(net, thr))
    try:
        alone = [pf.submit(q.ascii, q.offsets, r).future.result(timeout=120) for r, q in enumerate(reqs)]
        handles = [pf.submit(q.ascii, q.offsets, 100 + r) for r, q in enumerate(reqs)]
        mixed = [h.future.result(timeout=300) for h in handles]
    finally:
        pf.close()
    exact = [srv.submit(q.ascii, q.offsets, 200 + r).future.result(timeout=120) for r, q in enumerate(reqs)]
    kept = total = 0
    for a, m, x in zip(alone, mixed, exact):
        assert a.tobytes() == m.tobytes()
        ex = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(x["i"], x["j"]))}
        for rec in a:
            assert (int(rec["i"]), int(rec["j"])) in ex            # prefiltered edges are exact edges
            assert rec.tobytes() == x[ex[(int(rec["i"]), int(rec["j"]))]].tobytes()
        kept += len(a)
        total += len(x)
    assert 0 < kept <= total


def test_chunked_requests_equal_whole_requests(server):
    # requests split into chunks of 7 queries give the unsplit server's edges, alone
    # and all at once
    P, srv, db, reqs = server
    from paper_2009_14467_gb300 import serve as S
    whole = [srv.submit(q.ascii, q.offsets, 300 + r).future.result(timeout=300) for r, q in enumerate(reqs)]
    small = S.Server(db.ascii, db.offsets, P.Params(matrix=MAT), slots=3, reserve_bytes=1 << 30, chunk_queries=7)
    try:
        alone = [small.submit(q.ascii, q.offsets, r).future.result(timeout=300) for r, q in enumerate(reqs)]
        handles = [small.submit(q.ascii, q.offsets, 100 + r) for r, q in enumerate(reqs)]
        mixed = [h.future.result(timeout=300) for h in handles]
        st = small.latency_stats()
    finally:
        small.close()
    for w, a, m in zip(whole, alone, mixed):
        assert a.tobytes() == w.tobytes() and m.tobytes() == w.tobytes()
    assert st["requests"] == 2 * len(reqs)                 # one entry per request, not per chunk
