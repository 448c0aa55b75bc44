#!/usr/bin/env python
"""Benchmark of the PASTIS hot path on GB300: edges/s of the whole path a1..a10.

One step = encode -> k-mer matrix A -> substitute k-mers S -> A S -> candidates with
symmetrization -> Smith-Waterman of every candidate -> ANI/coverage filter, for one
batch: a block of query rows i of the synthetic protein set against every j > i (the
k-mer, S and AS stages run over the whole set in every step).  The row blocks split
the all-vs-all job into --batches parts of equal work, so the steps together cover the
whole job.  Inputs are resident in HBM.  The default workload is the 100,000-protein
planted-family set with 25 substitute k-mers and exact int32 SW.

Multi-GPU: the ranks split the row blocks of one job (rank r runs blocks r, r + N, ...);
each step is one block per rank, so per-GPU work per step is fixed ("weak" scaling) and
value = edges of all ranks / the slowest rank's time.  No data-path collective: the
blocks are independent given the replicated set.

`--impl reference` times the CPU oracle (oracle/) on host cores on bounded samples of
the same workload instead (the project's reference arm; no GPU work).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "edges/s (whole path: k-mers, A.S.A^T candidates, SW alignment, ANI/coverage filter)"
UNIT = "edges/s"
OPS_PER_CELL = 11          # integer ops per SW cell: E 3, F 3, H 4, running best 1
HALVES_PER_LANE = 2        # SW pass 1 works on 16-bit halves, two per 32-bit lane op
HALF_KINDS = ("viaddmax_s16x2", "vimax3_s16x2_relu", "vadd2", "max3_add2")   # 16x2 instructions
WORD_KINDS = ("iadd", "imax", "imad", "prmt")    # 32-bit kinds (the logic chain folds under the compiler)
SW1_DRAM_BYTES_PER_PAIR = 551_791_872 / 1_086_756

WORKLOADS = {
    "zipf_100k_s25_sw": dict(n=100_000, m=25, mode=3, desc=(
        "100,000 proteins: 10,000 Zipf(1.5, 1-200) families (80%) + 20% singletons, "
        "lengths log-normal(median 300) clipped 50-1000, 30% BLOSUM62 substitutions + 5% indels; "
        "k=6 with 25 substitute k-mers (C = A S A^T, symmetrized), min_shared 1, "
        "SW int32 BLOSUM62 open 11 / extend 1, ANI >= 30%, coverage >= 70%")),
    "zipf_20k_s25_sw": dict(n=20_000, m=25, mode=3, desc="20,000 proteins, same recipe (smaller stand-in)"),
    "zipf_5k_s25_sw": dict(n=5_000, m=25, mode=3, desc="5,000 proteins, same recipe (profiling stand-in)"),
    "zipf_1m_xd": dict(n=1_000_000, m=0, mode=4, desc=(
        "1,000,000 proteins: 100,000 Zipf(1.5, 1-200) families (80%) + 20% singletons, lengths log-normal"
        "(median 300) clipped 50-2000, same mutation recipe; k=6 exact k-mers, min_shared 1, x-drop (X = 49) "
        "from both seeds, BLOSUM62 open 11 / extend 1, ANI >= 30%, coverage >= 70%")),
    "zipf_20k_xd": dict(n=20_000, m=0, mode=4, desc=(
        "20,000 proteins of the 100,000-protein recipe; k=6 exact k-mers, x-drop (X = 49) from both seeds "
        "(profiling stand-in for the x-drop workloads)")),
    "families_1k_sw": dict(n=1000, m=0, mode=3, desc=(
        "1,000 proteins = 100 families x 10, k=6 exact, SW int32, ANI 30 / cov 70")),
}


def row_blocks(n, batches):
    """Query-row ranges [i0, i1) of equal all-vs-all work: row i pairs with n-1-i rows."""
    total = n * (n - 1) / 2.0
    bounds = [0]
    for k in range(1, batches):
        target = total * k / batches
        # work before row i: i*(n-1) - i*(i-1)/2; solve for i
        lo, hi = bounds[-1], n
        while lo < hi:
            mid = (lo + hi) // 2
            if mid * (n - 1) - mid * (mid - 1) / 2.0 < target:
                lo = mid + 1
            else:
                hi = mid
        bounds.append(lo)
    bounds.append(n)
    return [(bounds[k], bounds[k + 1]) for k in range(batches)]


def combine_ranks(my_ms, my_units, world, dist=None, device=None):
    """Max of the ranks' times and sum of their units (the bench's whole-job aggregate)."""
    if world <= 1 or dist is None:
        return my_ms, float(my_units)
    import torch
    t = torch.tensor([my_ms, float(my_units)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])


def rank_blocks(batches, world, rank):
    """The row blocks of one job that rank `rank` of `world` runs, in step order: blocks
    rank, rank + world, ... (every block goes to exactly one rank)."""
    return [b for b in range(batches) if b % world == rank]


def default_batches(n):
    return 64 if n >= 500_000 else 8 if n >= 50_000 else 1


def config_of(name, ps, batches, world):
    """The workload description both arms print (the same keys and values)."""
    return {"workload": WORKLOADS[name]["desc"], "name": name, "sequences": ps.n, "residues": int(ps.ascii.size),
            "batch": (f"one of {batches} equal-work query-row blocks (rows i against every j > i); "
                      f"the blocks together are the whole all-vs-all job"),
            "l2": "flushed between timed steps (512 MB write)", "parallelism": f"row blocks of one job split over {world} rank(s), no data-path collective"}


def make_set(name, seed_offset=0):
    w = WORKLOADS[name]
    if name.startswith("families_1k"):
        return synth.families_1k(seed=1 + seed_offset)
    if name == "zipf_1m_xd":
        return synth.zipf_1m(seed=3 + seed_offset)
    return synth.zipf_100k(seed=2 + seed_offset, n=w["n"])


# ---------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), power=float(f[3]),
                                 hw=f[5], hwt=f[6], swt=f[7], swp=f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows)}


# ---------------------------------------------------------------------------------
# CPU oracle on a bounded sample (the cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------------
def oracle_sample(ps, name, block, rng):
    """Runs the oracle's whole path on a block of random sequences of the set (every pair
    in a random block is a uniformly random pair of the set).  Returns (edges, seconds,
    pairs, cells)."""
    from oracle import oracle as O
    w = WORKLOADS[name]
    ids = np.sort(rng.choice(ps.n, size=min(block, ps.n), replace=False))
    sub = ps.subset(ids)
    t0 = time.perf_counter()
    r = O.run(sub.ascii, sub.offsets, synth.blosum62(), k=6, m=w["m"], mode=w["mode"])
    dt = time.perf_counter() - t0
    return len(r["edges"]), dt, len(ids) * (len(ids) - 1) // 2, r["cells"]


_POOL_SET = None


def _pool_init(asc, offs, name):
    global _POOL_SET
    _POOL_SET = (synth.ProteinSet(asc, offs, np.zeros(offs.size - 1, np.int32), name), name)


def _pool_block(job):
    seed, block = job
    ps, name = _POOL_SET
    return oracle_sample(ps, name, block, np.random.default_rng(seed))


class OraclePool:
    """The oracle on every host core: worker processes (spawn) each run the whole path on
    their own random block of the set; a round is one block per core, timed by the wall
    clock around it."""

    def __init__(self, ps, name):
        import multiprocessing as mp
        self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_pool_init,
                                                 initargs=(ps.ascii, ps.offsets, name))

    def round(self, block, seed):
        t0 = time.perf_counter()
        res = self.pool.map(_pool_block, [(seed + k, block) for k in range(self.cores)])
        dt = time.perf_counter() - t0
        return sum(r[0] for r in res), dt, sum(r[2] for r in res), sum(r[3] for r in res)

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    name = args.workload
    ps = make_set(name)
    block = args.ref_block
    pool = OraclePool(ps, name)
    for w_ in range(args.warmup):
        pool.round(block, 1000 * w_)
    edges = secs = pairs = cells = 0
    for st in range(args.steps):
        e, dt, p, c = pool.round(block, 12345 + 1000 * st)
        edges += e
        secs += dt
        pairs += p
        cells += c
    pool.close()
    value = edges / secs if secs > 0 else 0.0
    sample = (f"{args.steps} steps, each the oracle's whole path on {pool.cores} random blocks of {block} "
              f"sequences of the set in parallel, one per host core ({block * (block - 1) // 2} uniformly "
              f"random pairs per block); {pairs} pairs, {cells} DP cells, {edges} edges in {secs:.2f} s wall")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": config_of(name, ps, args.batches or default_batches(ps.n), max(1, args.gpus)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gcups": cells / secs / 1e9 if secs > 0 else 0.0}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------
# learned prefilter vs plain
# ---------------------------------------------------------------------------------
class PrefilterLeg:
    """The learned prefilter against the plain path on row blocks of one set: the MLP is
    trained on pass/fail labels of the exact path over one block, its threshold is
    calibrated for a recall target on another, and plain and prefiltered runs are timed
    on further blocks, with edge recall against the exact edges of the same blocks."""

    def __init__(self, P, F, ctx, a, o, params):
        self.P, self.F, self.ctx, self.a, self.o, self.params = P, F, ctx, a, o, params
        self.net = None
        self.thr = None

    def exact(self, rows):
        P, ctx, a, o, params = self.P, self.ctx, self.a, self.o, self.params
        codes = P.encode(ctx, a)
        A = P.build_kmers(ctx, codes, o, 6)
        cands = P.overlap_spgemm(ctx, A, params, rows=rows)
        alns = P.align_pairs(ctx, codes, o, cands, params)
        return codes, cands, alns

    def train(self, rows, train_pairs, seed=7):
        import torch
        F = self.F
        t0 = time.perf_counter()
        codes, cands, alns = self.exact(rows)
        y = F.labels_from(alns)
        x = F.features(self.ctx, codes, self.o, cands, self.params)
        n = x.shape[0]
        g = torch.Generator(device=x.device).manual_seed(seed)
        take = torch.randperm(n, device=x.device, generator=g)[:min(n, train_pairs)]
        xt, yt = x[take].contiguous(), y[take].contiguous()
        del codes, cands, alns, x, y
        self.net = F.MLP(seed=11)
        self.hist = F.train(self.ctx, self.net, xt, yt, epochs=3, batch=65536, lr=2e-3, seed=13)
        self.n_train = int(xt.shape[0])
        self.train_s = time.perf_counter() - t0

    def calibrate(self, rows, recall):
        F = self.F
        codes, cands, alns = self.exact(rows)
        yc = F.labels_from(alns)
        zc = F.forward(self.ctx, self.net, F.features(self.ctx, codes, self.o, cands, self.params))
        self.thr = F.threshold_for_recall(zc, yc, recall)

    def plain(self, rows):
        return self.P.run(self.ctx, self.a, self.o, self.params, rows=rows)

    def prefiltered(self, rows):
        P, F, ctx, a, o, params = self.P, self.F, self.ctx, self.a, self.o, self.params
        codes = P.encode(ctx, a)
        A = P.build_kmers(ctx, codes, o, 6)
        cands = P.overlap_spgemm(ctx, A, params, rows=rows)
        z = F.forward(ctx, self.net, F.features(ctx, codes, o, cands, params))
        kept = F.select(ctx, cands, z, self.thr)
        alns = P.align_pairs(ctx, codes, o, kept, params)
        edges = P.filter_edges(ctx, o, kept, alns, params)
        return dict(cands=cands, kept=kept, edges=edges)

    def compare(self, eval_blocks):
        import torch
        P = self.P

        def timed(fn):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.ctx.stream)
            out = fn()
            e1.record(self.ctx.stream)
            torch.cuda.synchronize()
            return out, e0.elapsed_time(e1) / 1000.0

        for rows in eval_blocks[:1]:          # warm-up of both forms
            self.plain(rows)
            self.prefiltered(rows)
        t_plain = t_pref = 0.0
        e_plain = e_pref = c_all = c_kept = missing = 0
        for rows in eval_blocks:
            rp, tp = timed(lambda: self.plain(rows))
            rf, tf = timed(lambda: self.prefiltered(rows))
            t_plain += tp
            t_pref += tf
            ep = P.to_records(rp["edges"], P.EDGE_DTYPE)
            ef = P.to_records(rf["edges"], P.EDGE_DTYPE)
            e_plain += len(ep)
            e_pref += len(ef)
            c_all += rp["cands"].shape[0]
            c_kept += rf["kept"].shape[0]
            kp = set(zip(ep["i"].tolist(), ep["j"].tolist()))
            missing += sum(1 for i, j in zip(ef["i"].tolist(), ef["j"].tolist()) if (i, j) not in kp)
        v_plain, v_pref = e_plain / t_plain, e_pref / t_pref
        return {"speedup": v_pref / v_plain, "edge_recall": e_pref / max(e_plain, 1),
                "edges_per_s_plain": v_plain, "edges_per_s_prefiltered": v_pref, "edges_not_in_exact": missing,
                "aligned_pair_reduction": 1.0 - c_kept / max(c_all, 1), "candidates": c_all, "kept": c_kept,
                "threshold": self.thr, "train_pairs": self.n_train, "train_s": round(self.train_s, 2),
                "train_loss": self.hist}


def start_set_generation(name):
    """Generates a set in a spawned process (started before the GPU work, so the set is
    ready when a later leg needs it).  Returns a future."""
    import concurrent.futures
    import multiprocessing as mp
    ex = concurrent.futures.ProcessPoolExecutor(1, mp_context=mp.get_context("spawn"))
    fut = ex.submit(make_set, name)
    ex.shutdown(wait=False)
    return fut


def xd_roofline(cells, ms, per_warp, half_rate, word_rate, n_sm, clk_mhz):
    """Roofline of the x-drop extensions' first phase for one launch of `cells` computed
    cells in `ms`: against the measured 16x2 peak when they run in 16-bit lanes
    (per_warp > 0), else the measured 32-bit peak."""
    achieved = cells * OPS_PER_CELL / (ms / 1000.0) / 1e12
    if per_warp:
        peak = n_sm * half_rate * 32 * HALVES_PER_LANE * clk_mhz * 1e6 / 1e12
        note = (f"measured: {n_sm} SMs x {half_rate:.3f} warp-instructions/clk/SM (best 16x2 kind of the probe) "
                f"x 32 lanes x {HALVES_PER_LANE} halves x {clk_mhz:.0f} MHz; 16-bit lanes, {per_warp} extensions per warp")
    else:
        peak = n_sm * word_rate * 32 * clk_mhz * 1e6 / 1e12
        note = (f"measured: {n_sm} SMs x {word_rate:.3f} warp-instructions/clk/SM (best 32-bit kind of the probe) "
                f"x 32 lanes x {clk_mhz:.0f} MHz; 32-bit lanes")
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "traffic": None, "kernel": "xd_extend", "peak_note": note, "ops_per_cell": OPS_PER_CELL,
            "cells": "computed cells of the x-drop extensions",
            "cells_per_clk_sm": cells / (ms / 1000.0) / (n_sm * clk_mhz * 1e6)}


def xd_leg(P, dev, half_rate, word_rate, n_sm, clk_mhz, n_blocks=2, pending=None, tune_pairs=1_000_000):
    """The 1,000,000-protein exact-k-mer x-drop configuration on a bounded sample: one
    warm-up row block, then `n_blocks` timed row blocks of its 64 (each the whole path:
    encode, A, candidates, x-drop alignment from both seeds, filter).  `pending`: the
    set's generation started earlier (start_set_generation), else it is generated here."""
    import torch
    name = "zipf_1m_xd"
    w = WORKLOADS[name]
    t0 = time.perf_counter()
    ps = pending.result() if pending is not None else make_set(name)
    gen_s = time.perf_counter() - t0
    params = P.Params(matrix=synth.blosum62(), k=6, m_subs=w["m"], mode=w["mode"])
    a = torch.from_numpy(ps.ascii).to(dev)
    o = torch.from_numpy(ps.offsets).to(dev)
    ctx = P.Context(dev.index or 0)
    batches = default_batches(ps.n)
    blocks = row_blocks(ps.n, batches)
    cells = torch.zeros(1, dtype=torch.int64, device=dev)
    r0 = P.run(ctx, a, o, params, rows=blocks[0])
    # extensions per warp, tuned on a sample of block 0's candidates (every stride-th query)
    cands0 = r0["cands"]
    stride = max(1, -(-cands0.shape[0] // tune_pairs))
    sample = cands0[(cands0.view(torch.int32).view(-1, 5)[:, 0] % stride) == 0].contiguous()
    pw, tms = P.autotune_xd(ctx, r0["codes"], o, sample, params, reps=2)
    del r0, cands0, sample
    torch.cuda.synchronize()
    ctx.profile(True)
    ms = 0.0
    edges = cands = 0
    for b in range(1, 1 + n_blocks):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        r = P.run(ctx, a, o, params, cells, rows=blocks[b])
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        edges += r["edges"].shape[0]
        cands += r["cands"].shape[0]
    prof = ctx.profile_read()
    ctx.profile(False)
    total_cells = int(cells.item())
    out = {"workload": w["desc"], "name": name, "sequences": ps.n,
           "blocks": f"row blocks 1-{n_blocks} of {batches} (block 0 as warm-up)",
           "edges_per_s": edges / (ms / 1000.0), "candidate_pairs_per_s": cands / (ms / 1000.0),
           "gcups": total_cells / (ms / 1000.0) / 1e9, "ms_per_block": ms / n_blocks,
           "candidates_per_block": cands // n_blocks, "edges_per_block": edges // n_blocks,
           "set_wait_s": round(gen_s, 1),
           "kernel_ms": {k: round(v[1], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])[:6]}}
    out["xd_per_warp"] = pw
    out["xd_tuner_ms"] = {("32-bit lanes" if c == 0 else f"16-bit lanes, {c} per warp"): round(v, 3)
                          for c, v in tms.items()}
    if "xd_extend" in prof:
        n_l, ms_l = prof["xd_extend"]
        out["roofline"] = xd_roofline(total_cells / max(1, n_l), ms_l / n_l, pw, half_rate, word_rate, n_sm, clk_mhz)
    ctx.close()
    return out


def run_prefilter(args):
    """Trains the MLP on pass/fail labels of the exact path over one row block of the
    100k set, calibrates the threshold for the recall target on a second block, then
    times plain vs prefiltered on further blocks and reports recall against the exact
    edges of the same blocks."""
    import torch
    import paper_2009_14467_gb300 as P
    from paper_2009_14467_gb300 import prefilter as F
    dev = torch.device("cuda", 0)
    name = args.workload
    w = WORKLOADS[name]
    ps = make_set(name)
    params = P.Params(matrix=synth.blosum62(), k=6, m_subs=w["m"], mode=w["mode"])
    a = torch.from_numpy(ps.ascii).to(dev)
    o = torch.from_numpy(ps.offsets).to(dev)
    ctx = P.Context(0)
    batches = args.batches or 16
    blocks = row_blocks(ps.n, batches)
    leg = PrefilterLeg(P, F, ctx, a, o, params)
    leg.train(blocks[0], args.train_pairs)
    src_desc = w["desc"]
    cal_rows, eval_from = blocks[1], 2
    if args.apply:
        # apply the trained network to a fresh set of another workload (e.g. the exact
        # k-mer x-drop pipeline of the 1,000,000-protein recipe, seed + 1)
        name = args.apply
        w = WORKLOADS[name]
        ps = make_set(name, seed_offset=1)
        leg.a = torch.from_numpy(ps.ascii).to(dev)
        leg.o = torch.from_numpy(ps.offsets).to(dev)
        leg.params = P.Params(matrix=synth.blosum62(), k=6, m_subs=w["m"], mode=w["mode"])
        batches = args.batches or (64 if ps.n >= 500_000 else 16)
        blocks = row_blocks(ps.n, batches)
        cal_rows, eval_from = blocks[0], 1
    leg.calibrate(cal_rows, args.calib_recall)
    eval_blocks = [blocks[k] for k in range(eval_from, min(batches, eval_from + max(args.steps, 1)))]
    r = leg.compare(eval_blocks)
    line = {"metric": "prefilter speedup vs plain at >= 99.5% edge recall (edges/s ratio)",
            "value": r["speedup"], "unit": "x", "higher_is_better": True, "n_gpus": 1,
            "steps": len(eval_blocks), "warmup": 1, "dtype": "bf16 (MLP) / int16x2 + int32 (alignment)", "data": "synthetic",
            "config": {"workload": w["desc"], "name": name, "batch": f"{len(eval_blocks)} of {batches} equal-work row blocks",
                       "train": (f"{r['train_pairs']} labelled candidates of block 0 of: {src_desc}, 3 epochs, Adam 2e-3"
                                 + (f"; applied to a fresh set (seed + 1) of {name}" if args.apply else "")),
                       "calibration": f"threshold {r['threshold']:.4f} for recall {args.calib_recall} on one block "
                                      f"(target {args.recall} on the evaluation blocks)"},
            "recall_target_met": r["edge_recall"] >= args.recall, **{k: v for k, v in r.items() if k != "speedup"}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# ---------------------------------------------------------------------------------
# variants of the graph (Sec. VI-B): components as families, CK threshold, NS weight
# ---------------------------------------------------------------------------------
def weighted_pr(labels, families):
    """Weighted precision (each cluster's largest family share) and recall (each
    family's largest cluster share) of a clustering, both over all proteins."""
    labels = np.asarray(labels, np.int64)
    families = np.asarray(families, np.int64)
    key = labels * (int(families.max()) + 1) + families
    k, cnt = np.unique(key, return_counts=True)
    lab_of, fam_of = k // (int(families.max()) + 1), k % (int(families.max()) + 1)
    best_l = np.zeros(int(labels.max()) + 1, np.int64)
    best_f = np.zeros(int(families.max()) + 1, np.int64)
    np.maximum.at(best_l, lab_of, cnt)
    np.maximum.at(best_f, fam_of, cnt)
    return float(best_l.sum()) / labels.size, float(best_f.sum()) / labels.size


def run_variants(args):
    """On the 20,000-protein set of the bench recipe (whole all-vs-all job per run):
    connected components of the ANI graph as protein families for m in {0, 10, 25, 50},
    scored by weighted precision / recall against the planted families (the paper's
    components table); the common-k-mer threshold t = 3 (min_shared 4) with 25
    substitutes; and the NS weight (score only, no traceback) against ANI at m = 25."""
    import torch
    from paper_2009_14467_gb300 import pastis as P
    dev = torch.device("cuda", 0)
    name = "zipf_20k_s25_sw"
    ps = make_set(name)
    a = torch.from_numpy(ps.ascii).to(dev)
    o = torch.from_numpy(ps.offsets).to(dev)
    ctx = P.Context(0)

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1000.0

    def ani_run(m, min_shared=1):
        params = P.Params(matrix=synth.blosum62(), k=6, m_subs=m, min_shared=min_shared)
        r = P.run(ctx, a, o, params)
        lab = P.components(ctx, ps.n, r["edges"])
        return r, lab

    rows = []
    ani_run(25)                                             # warm-up
    for m, ms in ((0, 1), (10, 1), (25, 1), (50, 1), (25, 4)):
        (r, lab), t = timed(lambda: ani_run(m, ms))
        prec, rec = weighted_pr(lab.cpu().numpy(), ps.family)
        rows.append({"m": m, "min_shared": ms, "candidates": int(r["cands"].shape[0]),
                     "edges": int(r["edges"].shape[0]), "components": int(np.unique(lab.cpu().numpy()).size),
                     "precision": round(prec, 4), "recall": round(rec, 4), "s": round(t, 3),
                     "edges_per_s": r["edges"].shape[0] / t})

    def ns_run():
        params = P.Params(matrix=synth.blosum62(), k=6, m_subs=25, mode=P.SW_SCORE)
        codes = P.encode(ctx, a)
        A = P.build_kmers(ctx, codes, o, 6)
        cands = P.overlap_spgemm(ctx, A, params)
        alns = P.align_pairs(ctx, codes, o, cands, params)
        return P.ns_edges(ctx, o, cands, alns)

    ns_run()
    e_ns, t_ns = timed(ns_run)
    ani25 = rows[2]
    line = {"metric": ("graph variants (Sec. VI-B) on 20,000 proteins: whole-job time with the ANI weight over "
                       "the NS weight at m = 25 (NS needs no traceback)"),
            "value": ani25["s"] / t_ns, "unit": "x", "higher_is_better": True,
            "n_gpus": 1, "steps": 1, "warmup": 1, "dtype": "int16x2 / int32", "data": "synthetic",
            "config": {"workload": WORKLOADS[name]["desc"] + "; whole all-vs-all job per run", "name": name},
            "components_as_families": rows,
            "ns": {"edges": int(e_ns.shape[0]), "s": round(t_ns, 3), "edges_per_s": e_ns.shape[0] / t_ns,
                   "weight": "score / shorter length, every pair with a positive score, no traceback"}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# ---------------------------------------------------------------------------------
# serving: query batches against a resident database
# ---------------------------------------------------------------------------------
def train_prefilter_net(P, F, ctx, dev, name, train_pairs, batches=16):
    """The prefilter network trained on pass/fail labels of the exact path over row
    block 0 of a set of the given workload (the same recipe as --mode prefilter)."""
    import torch
    w = WORKLOADS[name]
    ps = make_set(name)
    params = P.Params(matrix=synth.blosum62(), k=6, m_subs=w["m"], mode=w["mode"])
    a = torch.from_numpy(ps.ascii).to(dev)
    o = torch.from_numpy(ps.offsets).to(dev)
    t0 = time.perf_counter()
    codes = P.encode(ctx, a)
    A = P.build_kmers(ctx, codes, o, 6)
    cands = P.overlap_spgemm(ctx, A, params, rows=row_blocks(ps.n, batches)[0])
    alns = P.align_pairs(ctx, codes, o, cands, params)
    y = F.labels_from(alns)
    x = F.features(ctx, codes, o, cands, params)
    g = torch.Generator(device=dev).manual_seed(7)
    take = torch.randperm(x.shape[0], device=dev, generator=g)[:min(x.shape[0], train_pairs)]
    net = F.MLP(seed=11)
    hist = F.train(ctx, net, x[take].contiguous(), y[take].contiguous(), epochs=3, batch=65536, lr=2e-3, seed=13)
    return net, int(take.numel()), hist, time.perf_counter() - t0


def run_serve(args):
    """Database = the workload's protein set (exact k-mers, resident on the device).
    Requests of log-uniform 1..4096 queries (half drawn from the database's families,
    half from an unrelated set of the same recipe) arrive as a Poisson stream whose
    rate is 70% of the batch path's measured capacity; reports p50/p99 latency and
    queries/s of the server beside the plain batch path on the same queries."""
    import torch
    import paper_2009_14467_gb300 as P
    from paper_2009_14467_gb300 import serve as S
    name = args.workload
    w = WORKLOADS[name]
    db = make_set(name)
    # unrelated queries: a set of the same recipe with another seed (a 100,000-protein
    # one for the 1,000,000-protein database)
    other = make_set(name if db.n <= 100_000 else "zipf_100k_s25_sw", seed_offset=100)
    params = P.Params(matrix=synth.blosum62(), k=6, m_subs=0, mode=w["mode"])
    rng = np.random.default_rng(17)
    sizes = np.exp(rng.uniform(0.0, np.log(4096.0), size=args.requests)).astype(np.int64).clip(1, 4096)
    reqs = []
    for r, sz in enumerate(sizes):
        src = db if r % 2 == 0 else other
        reqs.append(src.subset(rng.choice(src.n, size=int(sz), replace=False)))
    pref = None
    if args.prefilter:
        # network trained on the 100k set's exact run; threshold calibrated for the recall
        # target on a separate batch of queries against this database
        from paper_2009_14467_gb300 import prefilter as F
        ctx = P.Context(0)
        net, n_train, hist, train_s = train_prefilter_net(P, F, ctx, torch.device("cuda", 0), "zipf_100k_s25_sw",
                                                          args.train_pairs)
        crng = np.random.default_rng(29)      # its own stream: the request stream stays the same
        cal = synth.from_strings([db.seq(int(i)) for i in crng.choice(db.n, 750, replace=False)] +
                                 [other.seq(int(i)) for i in crng.choice(other.n, 750, replace=False)])
        srv0 = S.Server(db.ascii, db.offsets, params, slots=1, reserve_bytes=8 << 30)
        cc = P.encode(ctx, torch.from_numpy(cal.ascii).cuda())
        co = torch.from_numpy(cal.offsets).cuda()
        cands = S.query_overlap(ctx, P.build_kmers(ctx, cc, co, 6), srv0.DB, params)
        alns = S.align_pairs_qt(ctx, cc, co, srv0.db_codes, srv0.db_offsets, cands, params)
        z = F.forward(ctx, net, F.features_qt(ctx, cc, co, srv0.db_codes, srv0.db_offsets, cands, params))
        thr = F.threshold_for_recall(z, F.labels_from(alns), args.calib_recall)
        srv0.close()
        ctx.close()
        pref = {"net": net, "threshold": thr, "train_pairs": n_train, "train_s": train_s,
                "calibration": f"threshold {thr:.4f} for recall {args.calib_recall} on 1,500 calibration queries"}
    srv = S.Server(db.ascii, db.offsets, params, slots=args.slots, reserve_bytes=8 << 30,
                   chunk_queries=args.chunk_queries)
    # warm-up, then the batch path: every request in turn on one slot, nothing overlapping
    for q in reqs[:3]:
        srv.submit(q.ascii, q.offsets).future.result()
    ctx = P.Context(0)

    def batch_path():
        """Every request in turn on one context; per-request times and edges."""
        times, n_e = [], 0
        torch.cuda.synchronize()
        t_all = time.perf_counter()
        for q in reqs:
            t1 = time.perf_counter()
            n_e += len(srv.process(ctx, S.Request(q.ascii, q.offsets, 0)))
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t1)
        return time.perf_counter() - t_all, n_e, np.array(times)

    graphs = None
    if args.no_graphs:
        srv.graphs = False
    else:
        # the same requests with the direct alignment call, for the graphs' effect
        srv.graphs = False
        batch_path()
        t_direct, _, times_direct = batch_path()
        srv.graphs = True
        batch_path()
    t_batch, n_edges_batch, times = batch_path()
    if not args.no_graphs:
        small = sizes <= 16
        graphs = {"alignment": "captured CUDA graph per worker context (pastis_align_plan)",
                  "batch_path_s_graphs": round(t_batch, 3), "batch_path_s_direct": round(t_direct, 3),
                  "median_request_ms_le16_queries_graphs": round(1e3 * float(np.median(times[small])), 3),
                  "median_request_ms_le16_queries_direct": round(1e3 * float(np.median(times_direct[small])), 3),
                  "requests_le16_queries": int(small.sum())}
    srv.drop_plan(ctx)
    ctx.close()
    nq = int(sizes.sum())
    cap = nq / t_batch
    rate = 0.7 * cap / float(sizes.mean())          # requests per second
    gaps = rng.exponential(1.0 / rate, size=len(reqs))
    srv.done.clear()
    handles = []
    t0 = time.perf_counter()
    for q, g in zip(reqs, gaps):
        time.sleep(g)
        handles.append(srv.submit(q.ascii, q.offsets))
    res_plain = [h.future.result(timeout=3600) for h in handles]
    n_edges = sum(len(r) for r in res_plain)
    st = srv.latency_stats()
    srv.close()
    pf = None
    if pref is not None:
        # the same stream through the prefilter: latency, throughput and edge recall
        srv = S.Server(db.ascii, db.offsets, params, slots=args.slots, reserve_bytes=8 << 30,
                       prefilter=(pref["net"], pref["threshold"]), chunk_queries=args.chunk_queries)
        for q in reqs[:3]:
            srv.submit(q.ascii, q.offsets).future.result()
        ctx = P.Context(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q in reqs:
            srv.process(ctx, S.Request(q.ascii, q.offsets, 0))
        torch.cuda.synchronize()
        cap_pf = nq / (time.perf_counter() - t0)
        srv.drop_plan(ctx)
        ctx.close()
        srv.done.clear()
        handles = []
        for q, g in zip(reqs, gaps):
            time.sleep(g)
            handles.append(srv.submit(q.ascii, q.offsets))
        res_pf = [h.future.result(timeout=3600) for h in handles]
        st_pf = srv.latency_stats()
        srv.close()
        kept = sum(len(r) for r in res_pf)
        outside = 0
        for a, x in zip(res_pf, res_plain):
            ex = set(zip(x["i"].tolist(), x["j"].tolist()))
            outside += sum(1 for i, j in zip(a["i"].tolist(), a["j"].tolist()) if (i, j) not in ex)
        pf = {"queries_per_s": st_pf["queries_per_s"], "p50_s": st_pf["p50_s"], "p99_s": st_pf["p99_s"],
              "batch_path_queries_per_s": cap_pf, "edges": kept, "edge_recall": kept / max(1, n_edges),
              "edges_not_in_exact": outside, "train_pairs": pref["train_pairs"], "train_s": pref["train_s"],
              "calibration": pref["calibration"]}
    line = {"metric": "serving: query batches vs a resident database (queries/s, p50/p99 latency)",
            "value": st["queries_per_s"], "unit": "queries/s", "higher_is_better": True, "n_gpus": 1,
            "steps": len(reqs), "warmup": 3, "data": "synthetic",
            "dtype": "int16x2 / int32" if w["mode"] not in (1, 4) else "int32",
            "config": {"workload": f"database: {w['desc']}; exact k-mers (m = 0)", "name": name,
                       "requests": len(reqs), "request_sizes": "log-uniform 1..4096 queries",
                       "arrivals": f"Poisson, {rate:.3f} requests/s (70% of batch capacity)",
                       "slots": args.slots, "chunk_queries": args.chunk_queries},
            "p50_s": st["p50_s"], "p99_s": st["p99_s"], "queries": nq,
            "batch_path_queries_per_s": cap, "edges": n_edges, "edges_batch_path": n_edges_batch,
            "graphs": graphs, "prefiltered": pf}
    print(json.dumps(line), flush=True)
    return 0 if n_edges == n_edges_batch else 1


# ---------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------
def run_probe(args):
    """The integer-pipe throughput probe alone: one line of warp-instructions per SM clock
    per instruction kind (the measured peak of the alignment roofline)."""
    import torch
    import paper_2009_14467_gb300 as P
    ctx = P.Context(0)
    rates = {k: max(P.probe_int_throughput(ctx, k, iters=args.probe_iters) for _ in range(2))
             for k in P.pastis.PROBE_KINDS}
    props = torch.cuda.get_device_properties(0)
    print(json.dumps({"probe": "integer-pipe throughput", "unit": "warp-instructions per SM clock",
                      "sms": props.multi_processor_count, "iters": args.probe_iters,
                      **{k: round(v, 4) for k, v in rates.items()}}), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="zipf_100k_s25_sw", choices=sorted(WORKLOADS))
    ap.add_argument("--ref-block", type=int, default=120)
    ap.add_argument("--batches", type=int, default=None,
                    help="equal-work query-row blocks the job is split into (default: 8 for 100k sets, else 1)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-prefilter", action="store_true", help="plain mode: skip the learned-prefilter leg")
    ap.add_argument("--no-xd-leg", action="store_true", help="plain mode: skip the 1M-protein x-drop leg")
    ap.add_argument("--no-graph-leg", action="store_true",
                    help="x-drop workloads: skip the block replayed from a captured CUDA graph")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default alignment layouts (no tuner)")
    ap.add_argument("--tune-pairs", type=int, default=3_000_000, help="candidates the tuner samples")
    ap.add_argument("--profile-json", default=None, help="write the per-kernel profile here")
    ap.add_argument("--probe-iters", type=int, default=20000, help="probe mode: loop iterations per kernel")
    ap.add_argument("--mode", default="plain", choices=["plain", "prefilter", "serve", "variants", "probe"],
                    help="plain: the exact path (the headline); prefilter: learned prefilter vs plain; "
                         "serve: query batches against a resident database; variants: components, CK, NS")
    ap.add_argument("--requests", type=int, default=48, help="serve mode: requests in the stream")
    ap.add_argument("--slots", type=int, default=4, help="serve mode: concurrent worker slots")
    ap.add_argument("--prefilter", action="store_true",
                    help="serve mode: also run the stream through the learned prefilter")
    ap.add_argument("--no-graphs", action="store_true", help="serve mode: direct alignment calls, no CUDA graphs")
    ap.add_argument("--chunk-queries", type=int, default=0,
                    help="serve mode: run requests above this many queries as chunks in rounds (0: whole)")
    ap.add_argument("--recall", type=float, default=0.995, help="edge recall the prefilter must keep")
    ap.add_argument("--calib-recall", type=float, default=0.998,
                    help="recall the threshold is calibrated for on the calibration block (margin over --recall)")
    ap.add_argument("--train-pairs", type=int, default=10_000_000)
    ap.add_argument("--apply", default=None, choices=sorted(WORKLOADS),
                    help="prefilter mode: evaluate the network trained on --workload on a fresh set of this workload")
    args = ap.parse_args()
    if args.warmup < 3:
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "prefilter":
        return run_prefilter(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "variants":
        return run_variants(args)
    if args.mode == "probe":
        return run_probe(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    xd_set = None
    if WORKLOADS[args.workload]["mode"] not in (1, 4) and not args.no_xd_leg and world == 1:
        xd_set = start_set_generation("zipf_1m_xd")       # ready by the time the x-drop leg runs

    import torch
    import torch.distributed as dist
    import paper_2009_14467_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    name = args.workload
    w = WORKLOADS[name]
    ps = make_set(name)                # one job; the ranks split its row blocks
    mat = synth.blosum62()
    params = P.Params(matrix=mat, k=6, m_subs=w["m"], mode=w["mode"])
    ascii_host = torch.from_numpy(ps.ascii).pin_memory()
    offs_host = torch.from_numpy(ps.offsets).pin_memory()
    ascii_dev = ascii_host.to(dev)
    offs_dev = offs_host.to(dev)
    ctx = P.Context(local_rank)
    cells = torch.zeros(1, dtype=torch.int64, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    batches = args.batches or default_batches(ps.n)
    if batches < world:
        batches = world
    blocks = row_blocks(ps.n, batches)
    mine = rank_blocks(batches, world, rank)
    counter = [0]

    def step():
        k = counter[0] % len(mine)
        counter[0] += 1
        if k == 0:
            # a new pass over this rank's share of the job: S and AS are built again
            # (the row blocks of one pass share them), so the steps carry their share
            ctx.forget()
        return P.run(ctx, ascii_dev, offs_dev, params, cells, rows=blocks[mine[k]])

    tune = None
    if w["mode"] not in (1, 4) and not args.no_autotune:
        # setup, untimed: the pass-1 layout per query-length bin, tuned on the candidates
        # of every stride-th query of block 0
        t0 = time.perf_counter()
        codes = P.encode(ctx, ascii_dev)
        A = P.build_kmers(ctx, codes, offs_dev, 6)
        cands = P.overlap_spgemm(ctx, A, params, rows=blocks[0])
        stride = max(1, -(-cands.shape[0] // args.tune_pairs))
        qi = cands.view(torch.int32).view(-1, 5)[:, 0]
        sample = cands[(qi % stride) == 0].contiguous()
        extra, cyc = P.autotune_sw(ctx, codes, offs_dev, sample, params, reps=2)
        torch.cuda.synchronize()
        base = float(cyc[0].sum())
        chosen = float(sum(cyc[extra[b], b] for b in range(P.pastis.SW_BINS)))
        tune = {"sample_pairs": int(sample.shape[0]), "sample": f"candidates of every {stride}th query of block 0",
                "setup_s": round(time.perf_counter() - t0, 2), "bins_changed": int((extra > 0).sum()),
                "layout": {f"{32 * b + 1}-{32 * b + 32}": ("int32 lanes" if extra[b] == P.pastis.SW_INT32
                                                            else f"+{int(extra[b])} stripes")
                           for b in np.flatnonzero(extra)},
                "int32_vs_int16_cycles": round(float(cyc[P.pastis.SW_INT32].sum()) / max(1.0, float(cyc[0].sum())), 3),
                "pass1_cycles_saved_on_sample": round(1.0 - chosen / base, 4) if base > 0 else 0.0}
        del codes, A, cands, qi, sample

    if w["mode"] == 4 and not args.no_autotune:
        # setup, untimed: x-drop extensions per warp (16-bit lanes) or 32-bit lanes, tuned
        # on the candidates of every stride-th query of block 0
        t0 = time.perf_counter()
        codes = P.encode(ctx, ascii_dev)
        A = P.build_kmers(ctx, codes, offs_dev, 6)
        cands = P.overlap_spgemm(ctx, A, params, rows=blocks[0])
        stride = max(1, -(-cands.shape[0] // args.tune_pairs))
        qi = cands.view(torch.int32).view(-1, 5)[:, 0]
        sample = cands[(qi % stride) == 0].contiguous()
        pw, tms = P.autotune_xd(ctx, codes, offs_dev, sample, params, reps=2)
        # the same timings per query-length bin of the sample (the setting is one per
        # batch; this shows whether any bin would choose otherwise)
        label = lambda c: "32-bit lanes" if c == 0 else f"16-bit lanes, {c} per warp"
        qlen = np.diff(ps.offsets)[sample.view(torch.int32).view(-1, 5)[:, 0].cpu().numpy()]
        by_bin = {}
        for lo, hi in ((50, 150), (150, 300), (300, 600), (600, 2001)):
            sel = torch.from_numpy(np.flatnonzero((qlen >= lo) & (qlen < hi))).to(dev)
            if sel.numel() == 0:
                continue
            bpw, bms = P.autotune_xd(ctx, codes, offs_dev, sample[sel].contiguous(), params, reps=2)
            by_bin[f"{lo}-{hi - 1}"] = {"pairs": int(sel.numel()), "fastest": label(min(bms, key=bms.get)),
                                        "ms": {label(c): round(v, 3) for c, v in bms.items()}}
        ctx.set_xd_layout(pw)
        torch.cuda.synchronize()
        tune = {"sample_pairs": int(sample.shape[0]), "sample": f"candidates of every {stride}th query of block 0",
                "setup_s": round(time.perf_counter() - t0, 2), "xd_per_warp": pw,
                "xd_ms_by_setting": {label(c): round(v, 3) for c, v in tms.items()},
                "by_query_length": by_bin}
        del codes, A, cands, qi, sample

    # the integer-pipe peak, measured on this GPU (warp-instructions per SM clock of each
    # instruction kind, the best of two runs): the alignment roofline divides by it
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    probe = {k: max(P.probe_int_throughput(ctx, k) for _ in range(2)) for k in P.PROBE_KINDS}

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)   # > L2 (129 MB)

    stream = ctx.stream
    clock = ClockSampler(local_rank)
    launches0 = ctx.launches
    ctx.profile(True)
    cells.zero_()
    step_ms = []
    edges_total = cands_total = 0
    clock.start()
    for _ in range(args.steps):
        flush.fill_(1)                 # evict the previous step's data from L2 (untimed)
        torch.cuda.synchronize()
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        res = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        step_ms.append(ev0.elapsed_time(ev1))
        edges_total += res["edges"].shape[0]
        cands_total += res["cands"].shape[0]
    clk = clock.stop()
    prof = ctx.profile_read()
    stats = ctx.stats()
    ctx.profile(False)
    launches = ctx.launches - launches0
    total_cells = int(cells.item())
    my_ms = sum(step_ms)
    max_ms, all_edges = combine_ranks(my_ms, edges_total, world, dist if world > 1 else None, dev)
    value = all_edges / (max_ms / 1000.0)

    # end to end through the public API from pinned host buffers (H2D + path + D2H)
    torch.cuda.synchronize()
    barrier()
    # the same row blocks as the timed steps, so both numbers cover the same work
    e2e_ms = []
    h2d = ascii_host.numel() + offs_host.numel() * 8
    d2h = 0
    e2e_edges = 0
    n_e2e = max(1, min(args.steps, 8))
    for k in range(n_e2e):
        flush.fill_(1)
        torch.cuda.synchronize()
        barrier()
        kb = (args.warmup + k) % len(mine)
        t0 = time.perf_counter()
        if kb == 0:
            ctx.forget()
        a = ascii_host.to(dev, non_blocking=True)
        o = offs_host.to(dev, non_blocking=True)
        r = P.run(ctx, a, o, params, rows=blocks[mine[kb]])
        edges_host = r["edges"].to("cpu")
        torch.cuda.synchronize()
        e2e_ms.append(1000 * (time.perf_counter() - t0))
        e2e_edges += edges_host.shape[0]
        d2h = edges_host.numel()
    e2e_t = torch.tensor([sum(e2e_ms)], dtype=torch.float64, device=dev)
    e2e_e = torch.tensor([float(e2e_edges)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)      # the slowest rank's time
        dist.all_reduce(e2e_e, op=dist.ReduceOp.SUM)      # every rank's edges
    e2e_value = float(e2e_e.item()) / (float(e2e_t.item()) / 1000.0)

    # roofline of the dominant kernel: SW pass 1 (integer-pipe bound).  Peak: the best
    # measured 16x2 instruction rate (warp-instructions per SM clock, from the probe) x 32
    # lanes x 2 halves x SMs x the SM clock sampled under load.
    roof = None
    dominant = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    clk_mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    half_rate = max(probe[k] for k in HALF_KINDS)
    word_rate = max(probe[k] for k in WORD_KINDS)
    probe_line = {"unit": "warp-instructions per SM clock (best of 2 runs, 4 CTAs x 256 threads per SM)",
                  **{k: round(v, 3) for k, v in probe.items()},
                  "sw_mix_cells_per_clk_sm": round(probe["sw_mix"] * 32 / 5.0, 2)}
    if "sw_pass1" in prof:
        n_l, ms_l = prof["sw_pass1"]
        per_launch_cells = total_cells / max(1, n_l)
        achieved = per_launch_cells * OPS_PER_CELL / (ms_l / n_l / 1000.0) / 1e12
        peak = n_sm * half_rate * 32 * HALVES_PER_LANE * clk_mhz * 1e6 / 1e12
        # DRAM bytes per launch: the ncu capture of this kernel on the 5,000-protein set of
        # the same recipe measured 551.8 MB for 1,086,756 pairs (the per-row-pair maxima
        # written for pass 2, which grow with the pairs), scaled by the launch's pairs
        traffic = SW1_DRAM_BYTES_PER_PAIR * cands_total / max(1, args.steps) if w["mode"] not in (1, 4) else None
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_note": "ncu DRAM bytes of a 5,000-protein launch scaled by pairs",
                "kernel": "sw_pass1",
                "peak_note": (f"measured: {n_sm} SMs x {half_rate:.3f} warp-instructions/clk/SM (best 16x2 kind "
                              f"of the probe) x 32 lanes x {HALVES_PER_LANE} halves x {clk_mhz:.0f} MHz"),
                "ops_per_cell": OPS_PER_CELL,
                "cells_per_clk_sm": per_launch_cells / (ms_l / n_l / 1000.0) / (n_sm * clk_mhz * 1e6),
                "recurrence_mix_cells_per_clk_sm": probe_line["sw_mix_cells_per_clk_sm"]}

    if "xd_extend" in prof and "sw_pass1" not in prof:
        # x-drop: the extensions' first phase, computed cells
        n_l, ms_l = prof["xd_extend"]
        roof = xd_roofline(total_cells / max(1, n_l), ms_l / n_l, ctx.xd_layout() if w["mode"] == 4 else 0,
                           half_rate, word_rate, n_sm, clk_mhz)
    # roofline of the overlap product (HBM bound): algorithmic bytes = 16 per left-operand
    # entry (its code, position and posting-list bounds), 8 per product (the posting
    # entry gathered), 20 per candidate record written
    roof_spg = None
    spg_ms = sum(v[1] for k, v in prof.items() if k.startswith("spgemm"))
    if spg_ms > 0 and stats["spgemm_products"] > 0:
        spg_bytes = 16 * stats["spgemm_left_entries"] + 8 * stats["spgemm_products"] + 20 * stats["spgemm_records"]
        peak_gbs, src = 6800.0, "fallback"
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peak_gbs, src = float(json.load(f)["hbm_gbs"]), "measured"
        except (OSError, KeyError, ValueError):
            pass
        ach = spg_bytes / (spg_ms / 1000.0) / 1e9
        roof_spg = {"bound": "hbm", "achieved": ach, "peak": peak_gbs, "unit": "GB/s", "frac": ach / peak_gbs,
                    "traffic": None, "kernel": "spgemm (cursors, rows, concat)", "peak_source": src,
                    "products": stats["spgemm_products"], "left_entries": stats["spgemm_left_entries"],
                    "records": stats["spgemm_records"]}
        # the same with the sorts that build A and AS counted as well: 8 bytes per element
        # per 8-bit digit pass, and the radix kernels' time
        sort_ms = sum(v[1] for k, v in prof.items() if k.startswith("radix"))
        if sort_ms > 0 and stats["sort_element_passes"] > 0:
            b2 = spg_bytes + 8 * stats["sort_element_passes"]
            a2 = b2 / ((spg_ms + sort_ms) / 1000.0) / 1e9
            roof_spg["with_sorts"] = {"achieved": a2, "frac": a2 / peak_gbs, "sort_element_passes":
                                      stats["sort_element_passes"], "sort_ms": sort_ms, "spgemm_ms": spg_ms}
    sw_block = None
    if w["mode"] in (1, 4) and rank == 0:
        # full SW over one block's candidates (the sample of the x-drop workload's pairs)
        sw_params = P.Params(matrix=mat, k=6, m_subs=w["m"], mode=0)
        codes = P.encode(ctx, ascii_dev)
        A = P.build_kmers(ctx, codes, offs_dev, 6)
        cands = P.overlap_spgemm(ctx, A, params, rows=blocks[0])
        del A
        c_sw = torch.zeros(1, dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.align_pairs(ctx, codes, offs_dev, cands, sw_params, c_sw)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1000.0
        sw_block = {"pairs": int(cands.shape[0]), "s": t, "pairs_per_s": cands.shape[0] / t,
                    "gcups": int(c_sw.item()) / t / 1e9,
                    "sample": "all candidates of row block 0 of the job (a fixed, seeded block of query rows)"}

    graph_leg = None
    if w["mode"] in (1, 4) and rank == 0 and not args.no_graph_leg:
        # the same block's x-drop alignment replayed from a captured CUDA graph (an
        # alignment plan: the whole set resident as targets, the block's rows as the query
        # batch) against the direct call: records equal, time of each
        def ev_time(fn):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return out, e0.elapsed_time(e1) / 1000.0

        i0, i1 = blocks[0]
        r0, r1 = int(ps.offsets[i0]), int(ps.offsets[i1])
        q_offs = (ps.offsets[i0:i1 + 1] - r0).astype(np.int64)
        q_pairs = cands.clone()
        q_pairs.view(torch.int32)[:, 0] -= i0                  # query index within the batch
        lmax = int(np.diff(ps.offsets).max())
        plan = P.AlignPlan(ctx, codes, offs_dev, params, i1 - i0, r1 - r0, int(cands.shape[0]), lmax)
        try:
            P.align_pairs(ctx, codes, offs_dev, cands, params)            # warm-up of both
            plan.run(codes[r0:r1], q_offs, q_pairs)
            direct, t_direct = ev_time(lambda: P.align_pairs(ctx, codes, offs_dev, cands, params))
            replay, t_graph = ev_time(lambda: plan.run(codes[r0:r1], q_offs, q_pairs))
            graph_leg = {"pairs": int(cands.shape[0]), "graph_nodes": plan.graph_nodes, "s_graph": t_graph,
                         "s_direct": t_direct, "records_equal": bool(torch.equal(replay, direct)),
                         "note": ("one graph launch per block (the plan copies the batch in and the records out) "
                                  "against the direct call's launches and synchronisations")}
        finally:
            plan.close()

    pref = None
    if w["mode"] not in (1, 4) and not args.no_prefilter and batches >= 5 and world == 1:
        # the learned prefilter against the plain path on this set (bounded: trained on
        # block 0, calibrated on block 1, timed on blocks 2 and 3)
        from paper_2009_14467_gb300 import prefilter as F
        del res
        leg = PrefilterLeg(P, F, ctx, ascii_dev, offs_dev, params)
        leg.train(blocks[0], args.train_pairs)
        leg.calibrate(blocks[1], args.calib_recall)
        pref = leg.compare([blocks[2], blocks[3]])
        pref.update({"recall_target": args.recall, "recall_target_met": pref["edge_recall"] >= args.recall,
                     "blocks": "trained on block 0, threshold calibrated on block 1 for recall "
                               f"{args.calib_recall}, timed on blocks 2 and 3 of the {batches}"})
        del leg

    xd = None
    if w["mode"] not in (1, 4) and not args.no_xd_leg and world == 1:
        # the 1,000,000-protein x-drop configuration, bounded to three row blocks
        xd = xd_leg(P, dev, half_rate, word_rate, n_sm, clk_mhz, pending=xd_set)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rng = np.random.default_rng(777)
        e1 = s1 = 0
        t_start = time.perf_counter()
        while time.perf_counter() - t_start < 8.0:
            de, dt, _, _ = oracle_sample(ps, name, args.ref_block, rng)
            e1 += de; s1 += dt
        pool = OraclePool(ps, name)
        e = s = p = c = 0
        r = 0
        while s < 12.0:
            de, dt, dp, dc = pool.round(args.ref_block, 777 + 1000 * r)
            e += de; s += dt; p += dp; c += dc; r += 1
        pool.close()
        cpu = {"value": e / s if s > 0 else 0.0, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
               "sample": (f"oracle whole path on random blocks of {args.ref_block} sequences of the same set, one "
                          f"block per host core in parallel ({pool.cores} processes): {p} uniformly random pairs, "
                          f"{c} DP cells, {e} edges in {s:.1f} s wall"),
               "single_core": {"value": e1 / s1 if s1 > 0 else 0.0, "edges": e1, "s": round(s1, 2)}}

    if rank == 0:
        kernel_ms = {k: round(v[1], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
        line = {
            "metric": METRIC if w["mode"] not in (1, 4) else METRIC.replace("SW alignment", "x-drop alignment"),
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "data": "synthetic",
            "dtype": "int16x2 (SW pass 1) / int32" if w["mode"] not in (1, 4) else "int32",
            "config": config_of(name, ps, batches, world),
            "gcups": total_cells / (my_ms / 1000.0) / 1e9,
            "candidate_pairs_per_s": cands_total / (my_ms / 1000.0),
            "candidates_per_step": cands_total // args.steps, "edges_per_step": edges_total // args.steps,
            "cells_per_step": total_cells // args.steps,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "roofline": roof, "roofline_spgemm": roof_spg, "dominant_kernel": dominant, "int_probe": probe_line,
            "kernel_ms_timed_region": kernel_ms,
            "sw_on_block": sw_block, "graph_on_block": graph_leg, "autotune": tune,
            "xdrop_1m": xd,
            "prefilter_speedup": pref["speedup"] if pref else None,
            "edge_recall": pref["edge_recall"] if pref else None, "prefilter": pref,
            "clocks": clk, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
        if args.profile_json:
            with open(args.profile_json, "w") as f:
                json.dump({"kernels": prof, "steps": args.steps, "cells": total_cells}, f, indent=1)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
