"""Host-side logic that needs no GPU: the prefilter's threshold choice, the bench's
clustering score against the oracle's, the alignment plan's capacity test, and the
synthetic generator's recipe (seeded, in range, the alphabet the path encodes)."""
import numpy as np
import pytest
import torch

import bench
import synth
from oracle import oracle as O


@pytest.mark.parametrize("seed,recall", [(0, 0.995), (1, 0.9), (2, 1.0), (3, 0.5)])
def test_threshold_keeps_the_recall_and_is_the_largest(seed, recall):
    from paper_2009_14467_gb300 import prefilter as F
    g = torch.Generator().manual_seed(seed)
    z = torch.randn(5000, generator=g)
    y = (torch.rand(5000, generator=g) < 0.3).float()
    thr = F.threshold_for_recall(z, y, recall)
    pos = z[y > 0.5]
    kept = (pos >= thr).float().mean().item()
    assert kept >= recall
    # any larger threshold among the positives' logits keeps too few
    above = pos[pos > thr]
    if above.numel():
        assert (pos >= above.min()).float().mean().item() < recall


def test_threshold_without_positives_keeps_everything():
    from paper_2009_14467_gb300 import prefilter as F
    assert F.threshold_for_recall(torch.randn(10), torch.zeros(10), 0.99) == float("-inf")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bench_clustering_score_equals_the_oracle(seed):
    rng = np.random.default_rng(seed)
    n = 3000
    fam = rng.integers(0, 200, size=n)
    lab = np.where(rng.random(n) < 0.7, fam * 3 + rng.integers(0, 2, size=n), rng.integers(0, 900, size=n))
    assert bench.weighted_pr(lab, fam) == pytest.approx(O.weighted_precision_recall(lab, fam), abs=1e-12)


def test_plan_capacity_test():
    from paper_2009_14467_gb300 import pastis as P
    plan = object.__new__(P.AlignPlan)             # the host-side test only, no device plan
    plan.max_q, plan.max_qres, plan.max_pairs, plan.max_len = 4, 100, 50, 40
    ok = np.array([0, 10, 50, 90], np.int64)
    assert plan.fits(ok, 50)
    assert not plan.fits(ok, 51)                                   # pairs
    assert not plan.fits(np.array([0, 10, 20, 30, 40, 50], np.int64), 1)   # queries
    assert not plan.fits(np.array([0, 41], np.int64), 1)          # a query too long
    assert not plan.fits(np.array([0, 40, 80, 101], np.int64), 1)  # residues
    plan.h = None                                                  # nothing to free


def test_generator_recipe():
    a, b = synth.families_1k(), synth.families_1k()
    assert a.ascii.tobytes() == b.ascii.tobytes()                  # seeded
    assert a.n == 1000 and np.bincount(a.family).tolist() == [10] * 100
    lens = np.diff(a.offsets)
    assert lens.min() >= 50 and lens.max() <= 1000
    letters = set(np.unique(a.ascii).tobytes().decode())
    assert letters <= set("ARNDCQEGHILKMFPSTWYV")                  # the 20 standard residues
    z = synth.zipf_100k(n=3000)
    zl = np.diff(z.offsets)
    assert z.n == 3000 and zl.min() >= 50 and zl.max() <= 1000
    sizes = np.bincount(z.family[z.family >= 0]) if (z.family >= 0).any() else np.array([])
    assert sizes.max() > 5 * np.median(sizes[sizes > 0])           # heavy-tailed family sizes


def test_serving_admission_by_memory():
    from paper_2009_14467_gb300.serve import ADMIT_WAIT_S, admissible
    G = 1 << 30
    assert admissible(free=40 * G, in_flight=10 * G, reserve=8 * G, need=20 * G, waited=0.0)
    assert not admissible(free=40 * G, in_flight=20 * G, reserve=8 * G, need=20 * G, waited=0.0)
    assert admissible(free=1 * G, in_flight=0, reserve=8 * G, need=20 * G, waited=0.0)      # alone
    assert admissible(free=1 * G, in_flight=5 * G, reserve=8 * G, need=20 * G, waited=ADMIT_WAIT_S + 0.01)


@pytest.mark.parametrize("n,chunk", [(1, 512), (512, 512), (513, 512), (4096, 512), (1000, 7), (10, 0)])
def test_serving_query_chunks_cover_in_order(n, chunk):
    from paper_2009_14467_gb300.serve import query_chunks
    r = query_chunks(n, chunk)
    assert r[0][0] == 0 and r[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))            # contiguous, in order
    sizes = [c1 - c0 for c0, c1 in r]
    assert min(sizes) >= 1
    if chunk > 0:
        assert max(sizes) <= chunk and max(sizes) - min(sizes) <= 1
    else:
        assert r == [(0, n)]


def test_reference_arm_prints_the_contract_line():
    # the reference arm is the oracle on the host cores: it runs without a GPU
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--workload", "families_1k_sw", "--ref-block", "40", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] >= 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_xd_roofline_peak_follows_the_lanes():
    """The x-drop roofline divides by the measured 16x2 peak when the extensions run in
    16-bit lanes and by the 32-bit peak otherwise; achieved = 11 ops per computed cell
    over the launch time."""
    cells, ms, n_sm, clk = 2.0e11, 500.0, 152, 2070.0
    half_rate, word_rate = 3.2, 3.9
    r16 = bench.xd_roofline(cells, ms, 4, half_rate, word_rate, n_sm, clk)
    r32 = bench.xd_roofline(cells, ms, 0, half_rate, word_rate, n_sm, clk)
    achieved = cells * bench.OPS_PER_CELL / (ms / 1000.0) / 1e12
    assert r16["achieved"] == pytest.approx(achieved) and r32["achieved"] == pytest.approx(achieved)
    assert r16["peak"] == pytest.approx(n_sm * half_rate * 32 * 2 * clk * 1e6 / 1e12)
    assert r32["peak"] == pytest.approx(n_sm * word_rate * 32 * clk * 1e6 / 1e12)
    assert r16["frac"] == pytest.approx(achieved / r16["peak"])
    assert "4 extensions per warp" in r16["peak_note"] and "32-bit lanes" in r32["peak_note"]
    assert r16["cells_per_clk_sm"] == pytest.approx(cells / (ms / 1000.0) / (n_sm * clk * 1e6))
