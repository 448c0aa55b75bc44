"""Pins for the oracle's Smith-Waterman, x-drop and filter: brute-force enumeration of
every alignment on short sequences, closed forms and invariants."""
import os

import numpy as np
import pytest

import synth
from oracle import oracle as O

A = synth.ALPHABET
MAT = synth.blosum62()
M = MAT.astype(int)


def _s(a, b):
    return int(M[A.index(a), A.index(b)])


def _enumerate_local(q, t, o, e):
    """Every local alignment that starts and ends with a residue pair:
    (score, qb, qe, tb, te, ident, cols), spans half-open.  A gap of length L costs
    o + (L-1)*e; a gap may follow a gap in the other sequence (a fresh open)."""
    out = []

    def rec(i, j, score, state, qb, tb, ident, cols):
        if state == "M":
            out.append((score, qb, i, tb, j, ident, cols))
        if i < len(q) and j < len(t):
            rec(i + 1, j + 1, score + _s(q[i], t[j]), "M", qb, tb, ident + (q[i] == t[j]), cols + 1)
        if i < len(q):
            rec(i + 1, j, score - (e if state == "F" else o), "F", qb, tb, ident, cols + 1)
        if j < len(t):
            rec(i, j + 1, score - (e if state == "E" else o), "E", qb, tb, ident, cols + 1)

    for i0 in range(len(q)):
        for j0 in range(len(t)):
            rec(i0 + 1, j0 + 1, _s(q[i0], t[j0]), "M", i0, j0, int(q[i0] == t[j0]), 1)
    return out


def _sw(q, t, o=11, e=1):
    ps = synth.from_strings([q, t])
    codes = O.encode(ps.ascii)
    pair = np.zeros(1, O.CAND_DTYPE)
    pair['i'], pair['j'], pair['count'] = 0, 1, 1
    rec, cells = O.align_pairs(codes, ps.offsets, pair, MAT, o, e, O.SW)
    return rec[0], cells


def _cases(seed, n, lo, hi, alphabet):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        yield (''.join(rng.choice(list(alphabet), size=int(rng.integers(lo, hi + 1)))),
               ''.join(rng.choice(list(alphabet), size=int(rng.integers(lo, hi + 1)))))


@pytest.mark.parametrize("o,e", [(11, 1), (3, 1), (2, 2), (1, 1)])
def test_sw_brute_force(o, e):
    # small gap costs make gapped optima and ties common
    for q, t in list(_cases(o * 7 + e, 14, 1, 6, "ACDWKS")) + [("WACW", "WCW"), ("AAAA", "AAAA")]:
        rec, cells = _sw(q, t, o, e)
        assert cells == len(q) * len(t)
        alns = _enumerate_local(q, t, o, e)
        best = max(a[0] for a in alns)
        if best <= 0:
            assert rec['score'] == 0 and rec['cols'] == 0 and rec['qe'] == 0
            continue
        assert rec['score'] == best
        opt = [a for a in alns if a[0] == best]
        got = (int(rec['qb']), int(rec['qe']), int(rec['tb']), int(rec['te']),
               int(rec['ident']), int(rec['cols']))
        assert got in {a[1:] for a in opt}
        # the end is the first maximum in row-major order
        first_end = min((a[2] - 1, a[4] - 1) for a in opt)
        assert (rec['qe'] - 1, rec['te'] - 1) == first_end


def test_sw_brute_force_length8():
    for q, t in _cases(99, 3, 8, 8, "ACWK"):
        t = t[:4]
        rec, _ = _sw(q, t)
        alns = _enumerate_local(q, t, 11, 1)
        best = max(a[0] for a in alns)
        assert rec['score'] == max(best, 0)


def test_sw_gap_convention_closed_form():
    # ten W against five W + AAA + five W: one gap of length 3 costs 11 + 2*1
    rec, _ = _sw("W" * 10, "W" * 5 + "AAA" + "W" * 5)
    assert rec['score'] == 10 * 11 - (11 + 2)
    assert rec['cols'] == 13 and rec['ident'] == 10
    assert (rec['qb'], rec['qe'], rec['tb'], rec['te']) == (0, 10, 0, 13)


def test_sw_single_residue_closed_forms():
    for a in A[:20]:
        for b in A[:20]:
            rec, _ = _sw(a, b)
            assert rec['score'] == max(0, _s(a, b))


def test_sw_self_score_and_symmetry():
    ps = synth.families_1k()
    rng = np.random.default_rng(5)
    for i in rng.choice(ps.n, 6, replace=False):
        s = ps.seq(int(i))[:200]
        rec, _ = _sw(s, s)
        assert rec['score'] == sum(_s(c, c) for c in s)
        assert rec['ident'] == rec['cols'] == len(s)
    for i, j in rng.choice(ps.n, (6, 2)):
        a, b = ps.seq(int(i))[:150], ps.seq(int(j))[:150]
        r1, _ = _sw(a, b)
        r2, _ = _sw(b, a)
        assert r1['score'] == r2['score'] >= 0


# ---- x-drop ------------------------------------------------------------------------

def _enumerate_prefix(q, t, o, e):
    """Best score over every alignment of a prefix of q with a prefix of t that starts
    at the anchor (0 for the empty one); no zero clamp."""
    best = [0]

    def rec(i, j, score, state):
        if state == "M" or (i, j) != (0, 0):
            best[0] = max(best[0], score)
        if i < len(q) and j < len(t):
            rec(i + 1, j + 1, score + _s(q[i], t[j]), "M")
        if i < len(q):
            rec(i + 1, j, score - (e if state == "F" else o), "F")
        if j < len(t):
            rec(i, j + 1, score - (e if state == "E" else o), "E")

    rec(0, 0, 0, "S")
    return best[0]


def _xd(q, t, qpos, tpos, k, X, o=11, e=1):
    ps = synth.from_strings([q, t])
    codes = O.encode(ps.ascii)
    pair = np.zeros(1, O.CAND_DTYPE)
    pair['i'], pair['j'], pair['count'] = 0, 1, 1
    pair['qpos'][0] = [qpos, 0xFFFF]
    pair['tpos'][0] = [tpos, 0xFFFF]
    rec, cells = O.align_pairs(codes, ps.offsets, pair, MAT, o, e, O.XD, X, k)
    return rec[0], cells


def test_xd_unbounded_is_prefix_alignment():
    # with X = infinity each extension is the best anchored prefix alignment
    for q, t in _cases(7, 12, 3, 7, "ACDWK"):
        k = 2
        qp, tp = 0, 0
        q2, t2 = q[:qp + k] + q[qp + k:], t
        rec, _ = _xd(q2, t2, qp, tp, k, 10 ** 6, 3, 1)
        seed = _s(q2[0], t2[0]) + _s(q2[1], t2[1])
        right = _enumerate_prefix(q2[k:], t2[k:], 3, 1)
        assert rec['score'] == seed + right


def test_xd_left_extension_unbounded():
    for q, t in _cases(8, 8, 3, 6, "ACDWK"):
        k = 2
        qq, tt = q + "WW", t + "WW"
        rec, _ = _xd(qq, tt, len(q), len(t), k, 10 ** 6, 3, 1)
        left = _enumerate_prefix(q[::-1], t[::-1], 3, 1)
        assert rec['score'] == left + 22


def test_xd_bounded_by_sw_and_self():
    ps = synth.families_1k()
    codes = O.encode(ps.ascii)
    rp, code, pos = O.kmers(codes, ps.offsets, 6)
    c = O.candidates(rp, code, pos, 6, 0, MAT, 1)[:300]
    sw, _ = O.align_pairs(codes, ps.offsets, c, MAT, mode=O.SW)
    xd, cells = O.align_pairs(codes, ps.offsets, c, MAT, mode=O.XD)
    assert (xd['score'] <= sw['score']).all()
    assert cells > 0
    s = ps.seq(3)
    rec, _ = _xd(s, s, 40, 40, 6, 49)
    assert rec['score'] == sum(_s(ch, ch) for ch in s)
    assert (rec['qb'], rec['qe'], rec['ident'], rec['cols']) == (0, len(s), len(s), len(s))


def test_xd_small_x_stops_early():
    # a strong seed followed by a long mismatching stretch: X smaller than the drop ends it
    q = "WWWWWW" + "PPPPPPPPPP" + "WWWWWW"
    t = "WWWWWW" + "GGGGGGGGGG" + "WWWWWW"
    big, _ = _xd(q, t, 0, 0, 6, 10 ** 6)
    small, _ = _xd(q, t, 0, 0, 6, 10)
    assert small['score'] == 66 and small['qe'] == 6
    assert big['score'] >= small['score']


# ---- filter -------------------------------------------------------------------------

def test_filter_boundaries():
    offs = np.array([0, 100, 200, 300], np.int64)     # lengths 100, 100, 100
    pairs = np.zeros(6, O.CAND_DTYPE)
    pairs['i'] = [0, 0, 0, 0, 0, 1]
    pairs['j'] = [1, 1, 1, 1, 1, 2]
    alns = np.zeros(6, O.ALN_DTYPE)
    # ANI exactly 30%, coverage exactly 70% on i -> kept (inclusive)
    alns[0] = (50, 0, 70, 0, 70, 30, 100, 0, 0, 0)
    # ANI 29/100 -> vetoed
    alns[1] = (50, 0, 70, 0, 70, 29, 100, 0, 0, 0)
    # coverage 69 -> vetoed
    alns[2] = (50, 0, 69, 0, 69, 30, 100, 0, 0, 0)
    # empty alignment -> never kept
    alns[3] = (0, 0, 0, 0, 0, 0, 0, 0, 0, 0)
    # equal lengths use sequence i: span on i is 70 although j only covers 10
    alns[4] = (50, 10, 80, 0, 10, 40, 80, 0, 0, 0)
    alns[5] = (50, 0, 100, 0, 100, 100, 100, 0, 0, 0)
    e = O.filter_edges(offs, pairs, alns)
    assert e['i'].tolist() == [0, 0, 1] and e['j'].tolist() == [1, 1, 2]
    assert e['weight'].tolist() == [np.float32(30) / np.float32(100), np.float32(40) / np.float32(80), 1.0]


def test_filter_uses_shorter_sequence():
    offs = np.array([0, 200, 300], np.int64)           # i has 200, j has 100
    pairs = np.zeros(2, O.CAND_DTYPE)
    pairs['j'] = 1
    alns = np.zeros(2, O.ALN_DTYPE)
    alns[0] = (50, 0, 50, 0, 70, 30, 80, 0, 0, 0)      # 70/100 on j: kept
    alns[1] = (50, 0, 150, 0, 69, 30, 80, 0, 0, 0)     # 69/100 on j: vetoed
    e = O.filter_edges(offs, pairs, alns)
    assert len(e) == 1



# ---- hand-worked x-drop cases (pruning with gaps, seed choice) ----------------------

_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "xdrop_worked.txt")


def _golden_matrix(name):
    """The scoring matrices the worked cases name (defined in the golden file)."""
    m = np.zeros((24, 24), np.int8)
    if name == "unit2":
        m[:] = -2
        np.fill_diagonal(m, 2)
    elif name == "cw":
        m[:] = -6
        for ch, v in (("C", 11), ("A", 4), ("D", 4), ("E", 4)):
            m[A.index(ch), A.index(ch)] = v
    else:
        raise ValueError(name)
    return m


def _golden_xd_cases():
    cases = []
    with open(_GOLDEN) as f:
        for line in f:
            tok = line.split("#", 1)[0].split()
            if not tok:
                continue
            assert tok[0] == "xd" and tok[9] == "->", line
            mat, (o, e, X, k), q, t = tok[1], map(int, tok[2:6]), tok[6], tok[7]
            seeds = [tuple(int(v) for v in s.split(":")) for s in tok[8].split(",")]
            cases.append((mat, o, e, X, k, q, t, seeds, tok[10:]))
    return cases


@pytest.mark.parametrize("case", _golden_xd_cases(), ids=lambda c: f"{c[5]}-{c[6]}-{c[7]}")
def test_xd_hand_worked(case):
    mat, o, e, X, k, q, t, seeds, want = case
    ps = synth.from_strings([q, t])
    codes = O.encode(ps.ascii)
    pair = np.zeros(1, O.CAND_DTYPE)
    pair['i'], pair['j'], pair['count'] = 0, 1, len(seeds)
    pair['qpos'][0] = [s[0] for s in seeds] + [0xFFFF] * (2 - len(seeds))
    pair['tpos'][0] = [s[1] for s in seeds] + [0xFFFF] * (2 - len(seeds))
    rec, cells = O.align_pairs(codes, ps.offsets, pair, _golden_matrix(mat), o, e, O.XD, X, k)
    r = rec[0]
    got = [int(r[f]) for f in ("score", "qb", "qe", "tb", "te", "ident", "cols", "seed_used", "passes")]
    assert got == [int(v) for v in want[:9]]
    if want[9] != "-":
        assert cells == int(want[9])


def test_filtered_mode_keeps_what_the_filter_needs():
    """Mode 3 (the filter only, Sec. IV-F): a passing pair's record is SW's, a failing
    pair keeps SW's score and end with the rest 0, and the edges are SW's."""
    ps = synth.zipf_100k(n=2000).subset(np.arange(150))
    codes = O.encode(ps.ascii)
    rp, code, pos = O.kmers(codes, ps.offsets, 6)
    c = O.candidates(rp, code, pos, 6, 10, MAT, 1)
    sw, cs = O.align_pairs(codes, ps.offsets, c, MAT, mode=O.SW)
    fl, cf = O.align_pairs(codes, ps.offsets, c, MAT, mode=O.SW_FILTERED)
    assert cs == cf
    ok = sw['passes'] == 1
    assert 0 < ok.sum() < len(c)
    assert fl[ok].tobytes() == sw[ok].tobytes()
    for f in ("score", "qe", "te"):
        assert (fl[f] == sw[f]).all()
    for f in ("qb", "tb", "ident", "cols", "passes"):
        assert (fl[f][~ok] == 0).all()
    assert O.filter_edges(ps.offsets, c, fl).tobytes() == O.filter_edges(ps.offsets, c, sw).tobytes()


def test_filtered_xd_mode_keeps_what_the_filter_needs():
    """Mode 4 (x-drop for the filter only): a passing pair's record is XD's, a failing
    pair keeps XD's score, end and seed with the rest 0, and the edges are XD's."""
    ps = synth.families_1k()
    codes = O.encode(ps.ascii)
    rp, code, pos = O.kmers(codes, ps.offsets, 6)
    c = O.candidates(rp, code, pos, 6, 0, MAT, 1)[:1500]
    xd, cx = O.align_pairs(codes, ps.offsets, c, MAT, mode=O.XD)
    fl, cf = O.align_pairs(codes, ps.offsets, c, MAT, mode=O.XD_FILTERED)
    assert cx == cf
    ok = xd['passes'] == 1
    assert 0 < ok.sum() < len(c)
    assert fl[ok].tobytes() == xd[ok].tobytes()
    for f in ("score", "qe", "te", "seed_used"):
        assert (fl[f] == xd[f]).all()
    for f in ("qb", "tb", "ident", "cols", "passes"):
        assert (fl[f][~ok] == 0).all()
    assert O.filter_edges(ps.offsets, c, fl).tobytes() == O.filter_edges(ps.offsets, c, xd).tobytes()
