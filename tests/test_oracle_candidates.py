"""Pins for the oracle's k-mer rows, substitute k-mers and candidate pairs against brute
force on small inputs (independent formulations: all-pairs set intersection, full
enumeration of the k-mer space, pairwise k-mer comparison)."""
import itertools

import numpy as np
import pytest

import synth
from oracle import oracle as O

A = synth.ALPHABET
MAT = synth.blosum62()


def _rand_set(rng, n, lo, hi, alphabet=A[:20]):
    return [''.join(rng.choice(list(alphabet), size=int(rng.integers(lo, hi + 1))))
            for _ in range(n)]


def _kmer_first_pos(s, k):
    """k-mer word -> first start (brute force over the string)."""
    d = {}
    for p in range(len(s) - k + 1):
        d.setdefault(s[p:p + k], p)
    return d


def _word_code(w):
    # the positional formula of Sec. V-B, written as a left-to-right Horner sum
    c = 0
    for ch in w:
        c = c * 24 + A.index(ch)
    return c


def _oracle_rows(strings, k):
    ps = synth.from_strings(strings)
    codes = O.encode(ps.ascii)
    return ps, codes, O.kmers(codes, ps.offsets, k)


@pytest.mark.parametrize("k", [1, 2, 3, 6])
def test_kmer_rows_brute(k):
    rng = np.random.default_rng(10 + k)
    strings = _rand_set(rng, 30, 0, 40, alphabet="ACDW") + ["A" * 20, "", "AC"[:k - 1] if k > 1 else ""]
    ps, codes, (rp, code, pos) = _oracle_rows(strings, k)
    for i, s in enumerate(strings):
        want = sorted((_word_code(w), p) for w, p in _kmer_first_pos(s, k).items())
        got = list(zip(code[rp[i]:rp[i + 1]].tolist(), pos[rp[i]:rp[i + 1]].tolist()))
        assert got == want


def _brute_exact(strings, k, min_shared=1):
    kms = [_kmer_first_pos(s, k) for s in strings]
    out = []
    for i, j in itertools.combinations(range(len(strings)), 2):
        shared = sorted(set(kms[i]) & set(kms[j]), key=_word_code)
        if len(shared) >= min_shared and shared:
            seeds = shared[:2]
            qp = [kms[i][w] for w in seeds] + [0xFFFF] * (2 - len(seeds))
            tp = [kms[j][w] for w in seeds] + [0xFFFF] * (2 - len(seeds))
            out.append((i, j, len(shared), tuple(qp), tuple(tp)))
    return out


def _as_tuples(c):
    return [(int(r['i']), int(r['j']), int(r['count']), tuple(int(x) for x in r['qpos']),
             tuple(int(x) for x in r['tpos'])) for r in c]


@pytest.mark.parametrize("seed,k,ms", [(0, 3, 1), (1, 2, 1), (2, 3, 2), (3, 4, 1), (4, 1, 3)])
def test_exact_candidates_brute(seed, k, ms):
    rng = np.random.default_rng(seed)
    strings = _rand_set(rng, 25, 0, 30, alphabet="ACDEW")
    ps, codes, (rp, code, pos) = _oracle_rows(strings, k)
    got = _as_tuples(O.candidates(rp, code, pos, k, 0, MAT, ms))
    assert got == _brute_exact(strings, k, ms)


def test_exact_candidates_invariants_family_set():
    ps = synth.families_1k().subset(np.arange(120))
    codes = O.encode(ps.ascii)
    rp, code, pos = O.kmers(codes, ps.offsets, 6)
    c = O.candidates(rp, code, pos, 6, 0, MAT, 1)
    assert (c['i'] < c['j']).all()
    keys = c['i'].astype(np.int64) * ps.n + c['j']
    assert (np.diff(keys) > 0).all()
    # swapping the two sequences mirrors the record
    for r in c[:20]:
        sub = ps.subset([r['j'], r['i']])
        cs = O.kmers(O.encode(sub.ascii), sub.offsets, 6)
        c2 = O.candidates(*cs, 6, 0, MAT, 1)
        assert len(c2) == 1 and c2[0]['count'] == r['count']
        assert list(c2[0]['qpos']) == list(r['tpos']) and list(c2[0]['tpos']) == list(r['qpos'])
    # count(i, i) would be the number of distinct k-mers: a sequence against its copy
    sub = ps.subset([5, 5])
    cs = O.kmers(O.encode(sub.ascii), sub.offsets, 6)
    c3 = O.candidates(*cs, 6, 0, MAT, 1)
    assert c3[0]['count'] == rp[6] - rp[5]


# ---- substitute k-mers -------------------------------------------------------------

def _all_codes_digits(k):
    n = 24 ** k
    codes = np.arange(n, dtype=np.int64)
    digits = np.zeros((n, k), dtype=np.int64)
    x = codes.copy()
    for t in range(k - 1, -1, -1):
        digits[:, t] = x % 24
        x //= 24
    return codes, digits


def _brute_nearest(root_digits, m, k, codes, digits):
    """The m k-mers q != r of least distance, ties by smaller code, by scanning the whole
    k-mer space."""
    M = MAT.astype(np.int64)
    expense = np.diag(M)[:, None] - M          # expense[a, b] = M[a,a] - M[a,b]
    d = np.zeros(codes.size, dtype=np.int64)
    for t in range(k):
        d += expense[root_digits[t], digits[:, t]]
    rcode = 0
    for t in range(k):
        rcode = rcode * 24 + int(root_digits[t])
    keep = codes != rcode
    order = np.lexsort((codes[keep], d[keep]))[:m]
    return codes[keep][order], d[keep][order], rcode


@pytest.mark.parametrize("k,m,nroots", [(1, 5, 24), (1, 23, 24), (2, 25, 576), (3, 25, 300), (3, 50, 100)])
def test_subkmers_full_enumeration(k, m, nroots):
    codes, digits = _all_codes_digits(k)
    rng = np.random.default_rng(k * 100 + m)
    roots = np.arange(24 ** k) if nroots >= 24 ** k else rng.choice(24 ** k, nroots, replace=False)
    sc, sd = O.subkmers(roots.astype(np.uint32), k, m, MAT)
    for r, root in enumerate(roots):
        wc, wd, rc = _brute_nearest(digits[root], m, k, codes, digits)
        assert sc[r, 0] == rc and sd[r, 0] == 0
        assert sc[r, 1:].tolist() == wc.tolist()
        assert sd[r, 1:].tolist() == wd.tolist()


def test_subkmers_k6_spot_roots():
    """k = 6: the distance of every one of the 24^6 k-mers from the root, as an outer
    sum over positions (C order of the array is the code order)."""
    k, m = 6, 25
    M = MAT.astype(np.int64)
    expense = np.diag(M)[:, None] - M
    for word in ["MKVLAT", "WWCHXY"]:
        root = [A.index(ch) for ch in word]
        d = np.zeros((1,) * k, dtype=np.int16)
        for t in range(k):
            shape = [1] * k
            shape[t] = 24
            d = d + expense[root[t]].astype(np.int16).reshape(shape)
        d = d.reshape(-1)
        rcode = _word_code(word)
        d[rcode] = np.iinfo(np.int16).max          # q != r
        want_c, want_d = [], []
        for D in range(int(d.min()), 200):
            idx = np.flatnonzero(d == D)           # ascending codes
            take = idx[:m - len(want_c)]
            want_c += take.tolist()
            want_d += [D] * len(take)
            if len(want_c) == m:
                break
        sc, sd = O.subkmers(np.array([rcode], np.uint32), k, m, MAT)
        assert sc[0, 1:].tolist() == want_c and sd[0, 1:].tolist() == want_d


def _brute_substitute_candidates(strings, k, m, min_shared):
    """Pairwise formulation of Sec. IV-C: the substitutes of i's k-mers that occur in j."""
    codes, digits = _all_codes_digits(k)
    kms = [_kmer_first_pos(s, k) for s in strings]
    srow = {}
    for w in set().union(*[set(x) for x in kms]):
        root = np.array([A.index(ch) for ch in w])
        wc, wd, rc = _brute_nearest(root, m, k, codes, digits)
        srow[rc] = {rc: 0, **{int(c): int(d) for c, d in zip(wc, wd)}}

    def oriented(i, j):
        kj = {_word_code(w): p for w, p in kms[j].items()}
        best = {}
        for w, p in kms[i].items():
            for q, d in srow[_word_code(w)].items():
                if q in kj:
                    cur = (d, p)
                    if q not in best or cur < best[q]:
                        best[q] = cur
        qs = sorted(best)
        return len(qs), [(best[q][1], kj[q]) for q in qs[:2]]

    out = []
    for i, j in itertools.combinations(range(len(strings)), 2):
        cf, sf = oriented(i, j)
        cb, sb = oriented(j, i)
        if cb > cf:
            cnt, seeds = cb, [(b, a) for a, b in sb]
        else:
            cnt, seeds = cf, sf
        if cnt >= min_shared and cnt > 0:
            qp = [s[0] for s in seeds] + [0xFFFF] * (2 - len(seeds))
            tp = [s[1] for s in seeds] + [0xFFFF] * (2 - len(seeds))
            out.append((i, j, cnt, tuple(qp), tuple(tp)))
    return out


@pytest.mark.parametrize("seed,k,m,ms", [(0, 2, 3, 1), (1, 3, 5, 1), (2, 3, 10, 2), (3, 2, 7, 3)])
def test_substitute_candidates_brute(seed, k, m, ms):
    rng = np.random.default_rng(100 + seed)
    strings = _rand_set(rng, 12, 0, 25, alphabet="ACDEKLSTW")
    ps, codes, (rp, code, pos) = _oracle_rows(strings, k)
    got = _as_tuples(O.candidates(rp, code, pos, k, m, MAT, ms))
    assert got == _brute_substitute_candidates(strings, k, m, ms)


def test_substitutes_m0_is_exact_and_monotone():
    ps = synth.families_1k().subset(np.arange(60))
    codes = O.encode(ps.ascii)
    rp, code, pos = O.kmers(codes, ps.offsets, 4)
    prev = None
    for m in [0, 2, 6]:
        c = O.candidates(rp, code, pos, 4, m, MAT, 1)
        keys = set(zip(c['i'].tolist(), c['j'].tolist()))
        if prev is not None:
            assert prev <= keys
        prev = keys
    exact = O.candidates(rp, code, pos, 4, 0, MAT, 1)
    assert _as_tuples(exact) == _brute_exact([ps.seq(i) for i in range(ps.n)], 4, 1)


# ---- hand-worked symmetrization -------------------------------------------------------

def _golden_sym_cases():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "symmetrize_worked.txt")
    cases = []
    with open(path) as f:
        for line in f:
            tok = line.split("#", 1)[0].split()
            if tok:
                assert tok[0] == "sym" and tok[6] == "->", line
                cases.append((tok[1], int(tok[2]), int(tok[3]), tok[4], tok[5], [int(v) for v in tok[7:]]))
    return cases


def _matrix_acd():
    m = np.full((24, 24), -4, np.int8)
    np.fill_diagonal(m, 5)
    for a, b, v in (("C", "C", 9), ("D", "D", 9), ("A", "C", 4), ("C", "D", 8)):
        m[A.index(a), A.index(b)] = m[A.index(b), A.index(a)] = v
    return m


@pytest.mark.parametrize("case", _golden_sym_cases(), ids=lambda c: f"{c[3]}-{c[4]}")
def test_symmetrization_hand_worked(case):
    mat, k, m, si, sj, want = case
    assert mat == "acd"
    ps, codes, (rp, code, pos) = _oracle_rows([si, sj], k)
    c = O.candidates(rp, code, pos, k, m, _matrix_acd(), 1)
    assert len(c) == 1 and (c[0]['i'], c[0]['j']) == (0, 1)
    assert [int(c[0]['count'])] + [int(v) for v in c[0]['qpos']] + [int(v) for v in c[0]['tpos']] == want
