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
