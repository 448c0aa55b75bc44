"""Parity at the benchmark's full sizes, in the launch configuration bench.py times:
the 100,000-protein set with 25 substitute k-mers and Smith-Waterman (one of 8
equal-work query-row blocks) and the 1,000,000-protein set with exact k-mers and x-drop
(one of 64 blocks), each in the bench's alignment mode (the filter-only forms).  The oracle cannot run these jobs whole, so outputs are sampled
and checked one by one:
 * candidate records: each sampled (i, j) against the oracle's product over the two
   sequences alone (a pair's semiring value depends on its two rows only);
 * completeness: for sampled rows, every j > i whose k-mers meet the row's (AS_i for
   substitutes: the first orientation) is a candidate;
 * alignments: sampled candidates aligned by the oracle;
 * edges: each sampled pair is an edge exactly when the oracle's filter keeps it, with
   the oracle's edge record."""
import numpy as np
import pytest
import torch

import bench
import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu
MAT = synth.blosum62()
N_SAMPLE = 300


@pytest.fixture(scope="module")
def P():
    from paper_2009_14467_gb300 import pastis
    return pastis


def _kmer_codes(codes, offsets, k):
    """Every k-mer of every sequence as (row, code) with code = sum c * 24^(k-1-q)."""
    n = offsets.size - 1
    L = codes.size
    W = max(0, L - k + 1)
    code = np.zeros(W, np.int64)
    for q in range(k):
        code = code * 24 + codes[q:W + q]
    lens = np.diff(offsets)
    row = np.repeat(np.arange(n, dtype=np.int32), lens)[:W]
    ok = np.arange(W) + k <= offsets[1:][row]                    # windows inside one sequence
    return row[ok], code[ok]


def _check(P, name, block, completeness_rows):
    w = bench.WORKLOADS[name]
    ps = bench.make_set(name)
    params = P.Params(matrix=MAT, k=6, m_subs=w["m"], mode=w["mode"])
    rows = bench.row_blocks(ps.n, 8 if ps.n < 500_000 else 64)[block]
    ctx = P.Context(0)
    try:
        res = P.run(ctx, torch.from_numpy(ps.ascii).cuda(), torch.from_numpy(ps.offsets).cuda(), params, rows=rows)
        cands = P.to_records(res["cands"], P.CAND_DTYPE)
        alns = P.to_records(res["alns"], P.ALN_DTYPE)
        edges = P.to_records(res["edges"], P.EDGE_DTYPE)
    finally:
        ctx.close()
    assert cands.size > 1_000_000 and (cands["i"] >= rows[0]).all() and (cands["i"] < rows[1]).all()
    assert (cands["j"] > cands["i"]).all()
    key = cands["i"].astype(np.int64) * ps.n + cands["j"]
    assert (np.diff(key) > 0).all()                               # (i, j) order, no repeats
    rng = np.random.default_rng(19)
    take = np.sort(rng.choice(cands.size, N_SAMPLE, replace=False))

    # candidate records, pair by pair
    for p in take:
        i, j = int(cands["i"][p]), int(cands["j"][p])
        two = ps.subset([i, j])
        c2 = O.encode(two.ascii)
        rp, code, pos = O.kmers(c2, two.offsets, 6)
        want = O.candidates(rp, code, pos, 6, w["m"], MAT, 1)
        assert want.size == 1
        got = cands[p:p + 1].copy()
        got["i"], got["j"] = 0, 1
        assert got.tobytes() == want.tobytes(), (i, j)

    # alignments and edges of the sampled pairs
    codes = O.encode(ps.ascii)
    want_a, _ = O.align_pairs(codes, ps.offsets, cands[take], MAT, mode=w["mode"])
    assert alns[take].tobytes() == want_a.tobytes()
    want_e = O.filter_edges(ps.offsets, cands[take], want_a)
    ekey = edges["i"].astype(np.int64) * ps.n + edges["j"]
    kept = {int(a) * ps.n + int(b): e.tobytes() for a, b, e in zip(want_e["i"], want_e["j"], want_e)}
    for p in take:
        kk = int(key[p])
        x = np.searchsorted(ekey, kk)
        present = x < ekey.size and ekey[x] == kk
        assert present == (kk in kept)
        if present:
            assert edges[x:x + 1].tobytes() == kept[kk]

    # completeness of sampled rows (first orientation)
    krow, kcode = _kmer_codes(codes, ps.offsets, 6)
    table = np.zeros(24 ** 6, np.bool_)
    for i in completeness_rows(rows, rng):
        mine = np.unique(kcode[krow == i])
        if w["m"] > 0:
            # the oracle's substitutes of the row's k-mers (its own code order: digits of
            # the first residue most significant, as here)
            subs, _ = O.subkmers(mine.astype(np.uint32), 6, w["m"], MAT)
            mine = np.unique(np.concatenate([mine, subs.astype(np.int64).ravel()]))
        table[:] = False
        table[mine] = True
        js = np.unique(krow[table[kcode]])
        js = js[js > i]
        have = cands["j"][cands["i"] == i]
        assert np.isin(js, have).all(), i
        if w["m"] == 0:
            assert np.array_equal(np.sort(have), js)                  # exact k-mers: the whole row


def test_fullsize_100k_substitutes_sw(P):
    _check(P, "zipf_100k_s25_sw", 3, lambda rows, rng: rng.integers(rows[0], rows[1], size=4))


def test_fullsize_1m_exact_xdrop(P):
    _check(P, "zipf_1m_xd", 3, lambda rows, rng: rng.integers(rows[0], rows[1], size=3))
