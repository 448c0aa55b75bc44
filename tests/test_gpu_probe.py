"""The integer-pipe probe that the alignment roofline divides by: every instruction kind
reports a rate no scheduler can exceed (4 warp-instructions per SM clock: one per
scheduler), the 16-bit maxima share one pipe (about 2 per clock), and mixing 16x2 maxima
with 16x2 adds, which run on different pipes, beats either alone."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import paper_2009_14467_gb300 as P
    ctx = P.Context(0)
    rates = {k: P.probe_int_throughput(ctx, k, iters=400) for k in P.PROBE_KINDS}
    yield P, ctx, rates
    ctx.close()


def test_rates_are_physical(env):
    _, _, rates = env
    for k, v in rates.items():
        assert 0.2 < v <= 4.1, (k, v)


def test_pipes(env):
    _, _, rates = env
    for k in ("viaddmax_s16x2", "vimax3_s16x2_relu", "imax"):
        assert 1.5 < rates[k] <= 2.1, (k, rates[k])
    assert rates["max3_add2"] > 1.2 * max(rates["vimax3_s16x2_relu"], rates["vadd2"])
    assert rates["iadd"] > 3.0


def test_bad_arguments_are_refused(env):
    P, ctx, _ = env
    out = ctypes.c_double()
    L = P.pastis.lib()
    assert L.pastis_probe_int_throughput(ctx.h, 99, 4, 10, ctypes.byref(out)) == 1     # unknown kind
    assert L.pastis_probe_int_throughput(ctx.h, 0, 0, 10, ctypes.byref(out)) == 1      # no CTAs
    assert L.pastis_probe_int_throughput(ctx.h, 0, 4, 0, ctypes.byref(out)) == 1       # no iterations
