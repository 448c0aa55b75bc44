"""Alignment plans: a batch's whole alignment captured once as a CUDA graph over
fixed-capacity buffers and replayed per batch.  Every record equals
pastis_align_pairs_qt's (and the oracle's on the combined set) for batches of different
sizes replayed on one graph, at the capacities, for an empty batch, and after batches
the plan refuses."""
import numpy as np
import pytest
import torch

import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu
MAT = synth.blosum62()
MAX_Q, MAX_PAIRS, MAX_LEN = 64, 6000, 1000


@pytest.fixture(scope="module")
def env():
    import paper_2009_14467_gb300 as P
    from paper_2009_14467_gb300 import serve as S
    ctx = P.Context(0)
    db = synth.families_1k()
    tcodes = P.encode(ctx, torch.from_numpy(db.ascii).cuda())
    toffs = torch.from_numpy(db.offsets).cuda()
    DB = P.build_kmers(ctx, tcodes, toffs, 6)
    yield P, S, ctx, db, tcodes, toffs, DB
    ctx.close()


def _batches():
    db = synth.families_1k()
    other = synth.families_1k(seed=9)
    rng = np.random.default_rng(33)
    out = []
    for r, size in enumerate([1, 7, 64, 20, 3]):
        src = db if r % 2 == 0 else other
        out.append(src.subset(rng.choice(src.n, size=size, replace=False)))
    return out


def _cands(P, S, ctx, q, DB, params):
    qc = P.encode(ctx, torch.from_numpy(q.ascii).cuda())
    qo = torch.from_numpy(q.offsets).cuda()
    c = S.query_overlap(ctx, P.build_kmers(ctx, qc, qo, 6), DB, params)
    return qc, qo, c[:MAX_PAIRS]


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
def test_plan_replays_equal_the_direct_call(env, mode):
    P, S, ctx, db, tcodes, toffs, DB = env
    params = P.Params(matrix=MAT, mode=mode)
    plan = P.AlignPlan(ctx, tcodes, toffs, params, MAX_Q, MAX_Q * MAX_LEN, MAX_PAIRS, MAX_LEN)
    try:
        assert plan.graph_nodes >= (5 if mode in (1, 4) else 9)   # memset, checks, the alignment kernels
        for r, q in enumerate(_batches()):
            qc, qo, c = _cands(P, S, ctx, q, DB, params)
            assert c.shape[0] > 0
            got = plan.run(qc, q.offsets, c)
            want = S.align_pairs_qt(ctx, qc, qo, tcodes, toffs, c, params)
            assert torch.equal(got, want), r
            if r == 2:
                # the oracle on [queries, targets], the query the row of each pair
                both = synth.from_strings([q.seq(i) for i in range(q.n)] + [db.seq(j) for j in range(db.n)])
                rec = P.to_records(c, P.CAND_DTYPE)
                rec["j"] += q.n
                ref, _ = O.align_pairs(O.encode(both.ascii), both.offsets, rec, MAT, mode=mode)
                assert P.to_records(got, P.ALN_DTYPE).tobytes() == ref.tobytes()
        # exactly the pair capacity (the batch's candidates repeated)
        q = _batches()[2]
        qc, qo, c = _cands(P, S, ctx, q, DB, params)
        full = c.repeat((MAX_PAIRS + c.shape[0] - 1) // c.shape[0], 1)[:MAX_PAIRS].contiguous()
        assert torch.equal(plan.run(qc, q.offsets, full),
                           S.align_pairs_qt(ctx, qc, qo, tcodes, toffs, full, params))
        # an empty batch
        assert plan.run(qc, q.offsets, full[:0]).shape[0] == 0
    finally:
        plan.close()


def test_plan_refuses_and_stays_usable(env):
    P, S, ctx, db, tcodes, toffs, DB = env
    params = P.Params(matrix=MAT)
    plan = P.AlignPlan(ctx, tcodes, toffs, params, MAX_Q, MAX_Q * MAX_LEN, MAX_PAIRS, MAX_LEN)
    try:
        q = _batches()[1]
        qc, qo, c = _cands(P, S, ctx, q, DB, params)
        want = S.align_pairs_qt(ctx, qc, qo, tcodes, toffs, c, params)
        over = c.repeat(MAX_PAIRS // c.shape[0] + 1, 1)[:MAX_PAIRS + 1].contiguous()
        with pytest.raises(P.PastisError) as e:
            plan.run(qc, q.offsets, over)
        assert e.value.status == 3                         # above the pair capacity
        bad = P.to_records(c, P.CAND_DTYPE)
        bad["j"][0] = db.n                                 # a target outside the set
        out = torch.full((c.shape[0], 20), 0xCD, dtype=torch.uint8, device="cuda")
        with pytest.raises(P.PastisError) as e:
            plan.run(qc, q.offsets, torch.from_numpy(bad.view(np.uint8).reshape(-1, 20)).cuda(), out=out)
        assert e.value.status == 1
        assert bool((out == 0xCD).all())                   # nothing written
        shifted = q.offsets + 1
        with pytest.raises(P.PastisError) as e:
            plan.run(qc, shifted, c)
        assert e.value.status == 1                         # offsets must start at 0
        long_q = synth.random_proteins(2, (MAX_LEN + 1, MAX_LEN + 50), seed=4)
        lc = P.encode(ctx, torch.from_numpy(long_q.ascii).cuda())
        with pytest.raises(P.PastisError) as e:
            plan.run(lc, long_q.offsets, c[:1])
        assert e.value.status == 3                         # a query longer than the plan admits
        # the next good batch gives the direct call's records
        assert torch.equal(plan.run(qc, q.offsets, c), want)
    finally:
        plan.close()


def test_plan_rejects_targets_it_cannot_hold(env):
    P, S, ctx, db, tcodes, toffs, DB = env
    with pytest.raises(P.PastisError) as e:
        P.AlignPlan(ctx, tcodes, toffs, P.Params(matrix=MAT), MAX_Q, MAX_Q * 100, MAX_PAIRS, 100)
    assert e.value.status == 1                             # targets longer than max_len
