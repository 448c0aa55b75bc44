"""Pins of the oracle's variant steps (Sec. VI-B): the score-only alignment mode, the NS
edge weight, connected components and the weighted precision / recall used to score
them against planted families."""
import numpy as np
import pytest

import synth
from oracle import oracle as O

MAT = synth.blosum62()


def _pairs(n):
    i, j = np.triu_indices(n, 1)
    c = np.zeros(i.size, O.CAND_DTYPE)
    c["i"], c["j"], c["count"] = i, j, 1
    return c


def test_score_mode_keeps_score_and_end_only():
    ps = synth.families_1k().subset(np.arange(40))
    codes = O.encode(ps.ascii)
    c = _pairs(ps.n)
    full, cells = O.align_pairs(codes, ps.offsets, c, MAT, mode=O.SW)
    sc, cells2 = O.align_pairs(codes, ps.offsets, c, MAT, mode=O.SW_SCORE)
    assert cells == cells2
    for f in ("score", "qe", "te"):
        assert (sc[f] == full[f]).all()
    for f in ("qb", "tb", "ident", "cols", "passes", "seed_used"):
        assert (sc[f] == 0).all()


def test_ns_weight_closed_form():
    # WCWCW against itself inside a longer target: score 11+9+11+9+11 = 51 over the
    # shorter sequence's 5 residues
    ps = synth.from_strings(["WCWCW", "GGWCWCWGGGGGGG"])
    codes = O.encode(ps.ascii)
    c = _pairs(2)
    alns, _ = O.align_pairs(codes, ps.offsets, c, MAT, mode=O.SW_SCORE)
    assert alns["score"][0] == 51
    e = O.ns_edges(ps.offsets, c, alns)
    assert e.size == 1 and e["weight"][0] == np.float32(10.2)
    # a pair with no positive cell is no edge
    ps2 = synth.from_strings(["WWWW", "PPPP"])
    a2, _ = O.align_pairs(O.encode(ps2.ascii), ps2.offsets, c, MAT, mode=O.SW_SCORE)
    assert a2["score"][0] == 0 and O.ns_edges(ps2.offsets, c, a2).size == 0


def _edges(pairs):
    e = np.zeros(len(pairs), O.EDGE_DTYPE)
    if len(pairs):
        e["i"], e["j"] = np.asarray(pairs).T
    return e


def test_components_hand_graph():
    lab = O.components(7, _edges([(5, 6), (1, 3), (3, 0), (4, 4)]))
    assert lab.tolist() == [0, 0, 2, 0, 4, 5, 5]
    assert O.components(3, _edges([])).tolist() == [0, 1, 2]
    with pytest.raises(ValueError):
        O.components(3, _edges([(0, 3)]))


def test_components_match_scipy():
    sp = pytest.importorskip("scipy.sparse")
    cg = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(5)
    for n, m in ((50, 30), (500, 400), (2000, 2500)):
        a = rng.integers(0, n, size=m)
        b = rng.integers(0, n, size=m)
        lab = O.components(n, _edges(list(zip(a, b))))
        g = sp.coo_matrix((np.ones(m), (a, b)), shape=(n, n))
        k, ref = cg.connected_components(g, directed=False)
        # same partition, and each label is the smallest vertex of its component
        first = {}
        for v, r in enumerate(ref.tolist()):
            first.setdefault(r, v)
        assert lab.tolist() == [first[r] for r in ref.tolist()]
        assert len(set(lab.tolist())) == k


def test_weighted_precision_recall_hand_cases():
    fam = [0, 0, 0, 1, 1]
    assert O.weighted_precision_recall([0, 0, 1, 1, 1], fam) == (0.8, 0.8)
    assert O.weighted_precision_recall([7, 7, 7, 7, 7], fam) == (0.6, 1.0)       # one cluster
    assert O.weighted_precision_recall([0, 1, 2, 3, 4], fam) == (1.0, 0.4)       # singletons
    assert O.weighted_precision_recall([3, 3, 3, 9, 9], fam) == (1.0, 1.0)       # exact
