"""Pins for the scoring input and the k-mer arithmetic against the paper's printed values
(tests/golden/paper_examples.txt) and the invariants the method relies on."""
import os

import numpy as np
import pytest

import synth
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.txt")
A = synth.ALPHABET


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for ln in f:
            ln = ln.split("#", 1)[0].strip()
            if ln:
                rows.append(ln.split())
    return rows


def _codes(s):
    return np.frombuffer(s.encode(), dtype=np.uint8)


def test_golden_file_has_every_kind():
    kinds = {r[0] for r in _golden()}
    assert kinds == {"kmer_id", "blosum", "match_score", "expense_row_prefix",
                     "substitute_distance", "closer_than_all"}


@pytest.mark.parametrize("row", [r for r in _golden() if r[0] == "kmer_id"])
def test_kmer_id_printed(row):
    # Sec. V-B worked example, through the oracle's own encode + k-mer step
    _, word, want = row
    codes = O.encode(_codes(word))
    rp, code, pos = O.kmers(codes, np.array([0, len(word)]), len(word))
    assert code.tolist() == [int(want)]
    assert pos.tolist() == [0]


def test_blosum_printed_values_and_invariants():
    m = synth.blosum62().astype(int)
    for r in _golden():
        if r[0] == "blosum":
            assert m[A.index(r[1]), A.index(r[2])] == int(r[3])
    assert (m == m.T).all()
    s = m[:20, :20]
    d = np.diag(s)
    assert (d > 0).all()
    # s(a,b) <= (s(a,a)+s(b,b))/2 on the standard block: needed for the self-score pin
    assert (2 * s <= d[:, None] + d[None, :]).all()
    assert m.max() == 11 and m[A.index("W"), A.index("W")] == 11
    p = synth.background()
    assert abs(p.sum() - 1.0) < 1e-6
    assert p @ s @ p < 0        # local alignment is meaningful only with E[score] < 0


@pytest.mark.parametrize("row", [r for r in _golden() if r[0] == "match_score"])
def test_match_scores_printed(row):
    m = synth.blosum62().astype(int)
    _, x, y, want = row
    assert sum(m[A.index(a), A.index(b)] for a, b in zip(x, y)) == int(want)


def test_expense_row_prefix_printed():
    m = synth.blosum62().astype(int)
    for r in _golden():
        if r[0] != "expense_row_prefix":
            continue
        a = A.index(r[1])
        row = sorted((m[a, a] - m[a, b], b) for b in range(24))  # ties by alphabet index
        for t, ent in enumerate(r[2:]):
            cost, base = ent.split(":")
            assert row[t] == (int(cost), A.index(base))


def test_substitute_examples_through_oracle_S():
    """Sec. IV-B: the printed distances, and the ordering claim, hold in the oracle's S."""
    mat = synth.blosum62()
    rows = _golden()
    root = "AAC"
    rc = O.kmers(O.encode(_codes(root)), np.array([0, 3]), 3)[1]
    # every 3-mer ranked by the oracle: m = 24^3 - 1 gives the whole order
    codes, dist = O.subkmers(rc, 3, 24 ** 3 - 1, mat)
    order = {int(c): t for t, c in enumerate(codes[0])}
    dmap = {int(c): int(d) for c, d in zip(codes[0], dist[0])}

    def code_of(w):
        return int(O.kmers(O.encode(_codes(w)), np.array([0, 3]), 3)[1][0])

    for r in rows:
        if r[0] == "substitute_distance":
            assert dmap[code_of(r[2])] == int(r[3])
        if r[0] == "closer_than_all":
            near = [code_of(w) for w in r[2].split(",")]
            prefix = r[3].rstrip("*")
            others = [code_of(prefix + b) for b in A if prefix + b != r[1]]
            assert max(order[c] for c in near) < min(order[c] for c in others)
            assert max(dmap[c] for c in near) < min(dmap[c] for c in others)


def test_encode_rejects_outside_alphabet():
    O.encode(_codes(A))
    for bad in ["a", "J", "O", "U", " ", "\n", "-"]:
        with pytest.raises(O.InvalidResidue):
            O.encode(_codes("AC" + bad + "D"))
    assert O.encode(_codes(A)).tolist() == list(range(24))
