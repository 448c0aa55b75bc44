"""The Smith-Waterman pass-1 layout (extra stripes, or 32-bit lanes, per query-length bin)
and its autotuner: every layout gives the same records as the default and the oracle, the
tuner returns and sets a valid layout, and bad layouts or modes are refused.  The same
for the x-drop lane layout's tuner (extensions per warp in 16-bit lanes)."""
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


def _families():
    ps = synth.families_1k()
    codes = O.encode(ps.ascii)
    rp, code, pos = O.kmers(codes, ps.offsets, 6)
    return ps, codes, O.candidates(rp, code, pos, 6, 0, MAT, 1)


def _long_pairs():
    # queries of 20..2100 residues (every bin, the last one past 2048), each against
    # five others, related pairs among them
    ps = synth.planted_families([6] * 12 + [3] * 10, 40, (20, 2100), seed=21)
    rng = np.random.default_rng(5)
    n = ps.n
    i = np.repeat(np.arange(n), 5)
    j = rng.integers(0, n, size=i.size)
    c = np.zeros(i.size, O.CAND_DTYPE)
    c["i"], c["j"], c["count"] = i, j, 1
    return ps, O.encode(ps.ascii), c


LAYOUTS = {
    "one": np.ones(64, np.uint8),
    "two": np.full(64, 2, np.uint8),
    "mixed": np.random.default_rng(3).integers(0, 3, size=64).astype(np.uint8),
    "int32": np.full(64, 3, np.uint8),
    "mixed_int32": np.random.default_rng(4).integers(0, 4, size=64).astype(np.uint8),
}


@pytest.mark.parametrize("mode", [0, 2])
def test_every_layout_gives_the_default_records(env, mode):
    P, ctx = env
    for ps, codes, c in (_families(), _long_pairs()):
        params = P.Params(matrix=MAT, mode=mode)
        ctx.set_sw_layout(None)
        base = P.to_records(P.align_pairs(ctx, dev(codes), dev(ps.offsets), recs(c), params), P.ALN_DTYPE)
        for name, lay in LAYOUTS.items():
            ctx.set_sw_layout(lay)
            assert np.array_equal(ctx.sw_layout(), lay)
            got = P.to_records(P.align_pairs(ctx, dev(codes), dev(ps.offsets), recs(c), params), P.ALN_DTYPE)
            assert got.tobytes() == base.tobytes(), name
        ctx.set_sw_layout(None)
        # the default against the oracle: the whole families set, a sample of the long pairs
        if ps.n == 1000:
            want, _ = O.align_pairs(codes, ps.offsets, c, MAT, mode=mode)
            assert base.tobytes() == want.tobytes()
        else:
            take = np.random.default_rng(9).choice(c.size, 60, replace=False)
            want, _ = O.align_pairs(codes, ps.offsets, c[take], MAT, mode=mode)
            assert base[take].tobytes() == want.tobytes()


def test_autotune_sets_a_valid_layout(env):
    P, ctx = env
    ps, codes, c = _long_pairs()
    params = P.Params(matrix=MAT)
    ctx.set_sw_layout(None)
    extra, cyc = P.autotune_sw(ctx, dev(codes), dev(ps.offsets), recs(c), params, reps=1)
    assert extra.shape == (64,) and set(np.unique(extra).tolist()) <= {0, 1, 2, P.SW_INT32}
    assert np.array_equal(ctx.sw_layout(), extra)
    assert cyc.shape == (4, 64) and (cyc >= 0).all()
    lens = np.diff(ps.offsets)
    bins = np.minimum(63, (lens[np.unique(c["i"])] - 1) // 32)
    for b in np.unique(bins):
        assert (cyc[:, b] > 0).all(), b              # every layout ran the bin's queries
    for b in np.setdiff1d(np.arange(64), bins):
        assert (cyc[:, b] == 0).all() and extra[b] == 0
    # a chosen layout is the fastest of the bin and beats the default by 2%
    for b in np.flatnonzero(extra):
        assert cyc[extra[b], b] == cyc[:, b].min() and cyc[extra[b], b] <= 0.98 * cyc[0, b]
    # the tuned context still gives the oracle's records
    take = np.random.default_rng(11).choice(c.size, 60, replace=False)
    got = P.to_records(P.align_pairs(ctx, dev(codes), dev(ps.offsets), recs(c[take]), params), P.ALN_DTYPE)
    want, _ = O.align_pairs(codes, ps.offsets, c[take], MAT)
    assert got.tobytes() == want.tobytes()
    ctx.set_sw_layout(None)


def test_bad_layouts_and_modes_are_refused(env):
    P, ctx = env
    ctx.set_sw_layout(LAYOUTS["one"])
    bad = np.zeros(64, np.uint8)
    bad[17] = P.SW_INT32 + 1
    with pytest.raises(P.PastisError) as e:
        ctx.set_sw_layout(bad)
    assert e.value.status == 1
    assert np.array_equal(ctx.sw_layout(), LAYOUTS["one"])     # unchanged
    ps, codes, c = _families()
    with pytest.raises(P.PastisError) as e:
        P.autotune_sw(ctx, dev(codes), dev(ps.offsets), recs(c[:100]), P.Params(matrix=MAT, mode=P.XD))
    assert e.value.status == 7
    assert np.array_equal(ctx.sw_layout(), LAYOUTS["one"])
    ctx.set_sw_layout(None)
    assert (ctx.sw_layout() == 0).all()


def test_xd_autotune_sets_a_valid_setting(env):
    """The x-drop lane tuner: times every setting, sets the fastest (or keeps the current
    one within 2%), and the tuned context still gives the oracle's mode-4 records."""
    P, ctx = env
    ps, codes, c = _families()
    params = P.Params(matrix=MAT, mode=P.XD_FILTERED)
    ctx.set_xd_layout()
    pw, ms = P.autotune_xd(ctx, dev(codes), dev(ps.offsets), recs(c), params, reps=2)
    assert pw in P.XD_CHOICES and ctx.xd_layout() == pw
    assert set(ms) == set(P.XD_CHOICES) and all(v > 0 for v in ms.values())
    if pw != P.XD_DEFAULT_PER_WARP:
        assert ms[pw] == min(ms.values()) and ms[pw] <= 0.98 * ms[P.XD_DEFAULT_PER_WARP]
    got = P.to_records(P.align_pairs(ctx, dev(codes), dev(ps.offsets), recs(c), params), P.ALN_DTYPE)
    want, _ = O.align_pairs(codes, ps.offsets, c, MAT, mode=P.XD_FILTERED)
    assert got.tobytes() == want.tobytes()
    # the SW modes are refused and the setting stays
    with pytest.raises(P.PastisError) as e:
        P.autotune_xd(ctx, dev(codes), dev(ps.offsets), recs(c[:100]), P.Params(matrix=MAT, mode=P.SW))
    assert e.value.status == 7
    assert ctx.xd_layout() == pw
    ctx.set_xd_layout()
