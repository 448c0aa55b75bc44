"""GPU parity: every step of the CUDA path against the CPU oracle, bit-exact (all work is
integer; the one float, the edge weight, is a correctly rounded quotient on both sides).
Sizes span several tiles, stripes and ragged tails; edge cases cover empty and short
sequences, repeats and the degenerate alignments."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu

MAT = synth.blosum62()


@pytest.fixture(scope="module")
def P():
    import paper_2009_14467_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(P):
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    c = P.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def edge_case_set():
    strings = ["", "A", "ACDEF", "ACDEFG", "AAAAAAAAAAAAAAAAAAAA", "WWWWWWW", "ACDEFGACDEFGACDEFG",
               "MKV" * 40, "", "GGGGGGGGGGGGGGGGGGGGGGGGGGGGGGG", "ACDEFGHIKLMNPQRSTVWY" * 3]
    rng = np.random.default_rng(7)
    strings += [''.join(rng.choice(list(synth.ALPHABET[:20]), size=int(rng.integers(0, 300))))
                for _ in range(40)]
    return synth.from_strings(strings)


# ---- a1 ------------------------------------------------------------------------------

def test_encode_parity_and_errors(P, ctx):
    ps = synth.families_1k()
    got = P.encode(ctx, dev(ps.ascii)).cpu().numpy()
    assert (got == O.encode(ps.ascii)).all()
    # unaligned view and ragged tail
    sub = dev(ps.ascii)[3:3 + 1001]
    assert (P.encode(ctx, sub).cpu().numpy() == O.encode(ps.ascii[3:1004])).all()
    bad = ps.ascii.copy()
    bad[777] = ord("a")
    bad[9000] = ord("J")
    with pytest.raises(P.PastisError) as e:
        P.encode(ctx, dev(bad))
    assert e.value.status == 2 and "777" in str(e.value)


# ---- a2-a3 ---------------------------------------------------------------------------

def _oracle_csc(rp, code, pos, n, k):
    seq = np.repeat(np.arange(n, dtype=np.int32), np.diff(rp))
    order = np.lexsort((seq, code))
    counts = np.bincount(code, minlength=24 ** k)
    col_ptr = np.zeros(24 ** k + 1, np.int64)
    np.cumsum(counts, out=col_ptr[1:])
    return col_ptr, seq[order], pos[order]


@pytest.mark.parametrize("which,k", [("families", 6), ("families", 3), ("edge", 6), ("edge", 2), ("edge", 1)])
def test_build_kmers_parity(P, ctx, which, k):
    ps = synth.families_1k() if which == "families" else edge_case_set()
    codes = O.encode(ps.ascii)
    rp, code, pos = O.kmers(codes, ps.offsets, k)
    A = P.build_kmers(ctx, dev(codes), dev(ps.offsets), k)
    assert A.nnz == code.size
    assert (A.row_ptr.cpu().numpy() == rp).all()
    assert (A.row_code[:A.nnz].cpu().numpy().view(np.uint32) == code).all()
    assert (A.row_pos[:A.nnz].cpu().numpy().view(np.uint16) == pos).all()
    cp, cs, cpos = _oracle_csc(rp, code, pos, ps.n, k)
    assert (A.col_ptr.cpu().numpy().view(np.uint32).astype(np.int64) == cp).all()
    assert (A.col_seq[:A.nnz].cpu().numpy() == cs).all()
    assert (A.col_pos[:A.nnz].cpu().numpy().view(np.uint16) == cpos).all()


# ---- a4 ------------------------------------------------------------------------------

@pytest.mark.parametrize("k,m", [(6, 25), (6, 50), (3, 25), (2, 40), (1, 23), (6, 128)])
def test_substitute_kmers_parity(P, ctx, k, m):
    rng = np.random.default_rng(k * 1000 + m)
    roots = rng.choice(24 ** k, size=min(3000, 24 ** k), replace=False).astype(np.uint32)
    # include roots made of the odd symbols (negative expenses for X, B/Z ties, *)
    extra = [sum(c * 24 ** (k - 1 - t) for t, c in enumerate(w[:k]))
             for w in ([22] * 6, [20, 21, 22, 23, 22, 20], [23] * 6, [4] * 6, [17] * 6)]
    roots = np.unique(np.concatenate([roots, np.array(extra, np.uint32)]))
    want_c, want_d = O.subkmers(roots, k, m, MAT)
    gc, gd = P.substitute_kmers(ctx, dev(roots.view(np.int32)), P.Params(matrix=MAT, k=k, m_subs=m))
    assert (gc.cpu().numpy().view(np.uint32) == want_c).all()
    assert (gd.cpu().numpy() == want_d).all()


# ---- a5-a7 ---------------------------------------------------------------------------

def _cands(P, ctx, ps, k=6, m=0, min_shared=1):
    codes = O.encode(ps.ascii)
    A = P.build_kmers(ctx, dev(codes), dev(ps.offsets), k)
    got = P.to_records(P.overlap_spgemm(ctx, A, P.Params(matrix=MAT, k=k, m_subs=m, min_shared=min_shared)),
                       P.CAND_DTYPE)
    rp, code, pos = O.kmers(codes, ps.offsets, k)
    want = O.candidates(rp, code, pos, k, m, MAT, min_shared)
    return got, want


@pytest.mark.parametrize("min_shared", [1, 2, 4])
def test_candidates_exact_parity(P, ctx, min_shared):
    got, want = _cands(P, ctx, synth.families_1k(), min_shared=min_shared)
    assert len(got) == len(want)
    assert got.tobytes() == want.tobytes()


def test_candidates_exact_edge_cases(P, ctx):
    ps = edge_case_set()
    for k in (1, 2, 6):
        got, want = _cands(P, ctx, ps, k=k)
        assert got.tobytes() == want.tobytes()


def test_candidates_split_rows(P, ctx):
    # many copies of one family: rows with many partners, tables up to their limit
    fam = synth.planted_families([700], 0, (60, 120), seed=11)
    got, want = _cands(P, ctx, fam, k=3)
    assert got.tobytes() == want.tobytes()


def _shared_kmer_set():
    # 4,400 sequences holding one common 6-mer (WWWWWW, W nowhere else) among 20,000
    # unrelated ones: the first rows have more distinct partners than a table holds,
    # all of them in the first column range the product bound suggests, so the row
    # takes several ranges and the first ones overflow and are halved
    rng = np.random.default_rng(1)
    alpha = np.frombuffer(b"ARNDCQEGHILKMFPSTYV", dtype=np.uint8)
    rnd = lambda n: rng.choice(alpha, n).tobytes().decode()
    strs = ["WWWWWW" + rnd(20)] + [rnd(10) + "WWWWWW" + rnd(10) for _ in range(4400)]
    strs += [rnd(30) for _ in range(20000)]
    return synth.from_strings(strs)


@pytest.mark.parametrize("m", [0, 3])
def test_candidates_rows_in_column_ranges(P, ctx, m):
    got, want = _cands(P, ctx, _shared_kmer_set(), k=6, m=m)
    assert len(want) > 9_000_000
    assert len(got) == len(want)
    assert got.tobytes() == want.tobytes()


@pytest.mark.parametrize("m,min_shared,k", [(25, 1, 6), (10, 4, 6), (5, 1, 4)])
def test_candidates_substitute_parity(P, ctx, m, min_shared, k):
    ps = synth.zipf_100k(n=2000).subset(np.arange(300))
    got, want = _cands(P, ctx, ps, k=k, m=m, min_shared=min_shared)
    assert len(got) == len(want)
    assert got.tobytes() == want.tobytes()


def test_spgemm_capacity_protocol(P, ctx):
    ps = synth.families_1k().subset(np.arange(200))
    codes = O.encode(ps.ascii)
    A = P.build_kmers(ctx, dev(codes), dev(ps.offsets), 6)
    p = P.Params(matrix=MAT).c()
    nout = ctypes.c_int64()
    st = P.pastis.lib().pastis_overlap_spgemm(ctx.h, ctypes.byref(A.c()), ctypes.byref(p), None, 0,
                                                ctypes.byref(nout))
    assert st == 3 and nout.value > 0
    out = torch.empty((nout.value, 20), dtype=torch.uint8, device="cuda")
    st = P.pastis.lib().pastis_overlap_spgemm(ctx.h, ctypes.byref(A.c()), ctypes.byref(p),
                                                ctypes.c_void_p(out.data_ptr()), nout.value, ctypes.byref(nout))
    assert st == 0


# ---- a8-a10 --------------------------------------------------------------------------

def _align_both(P, ctx, ps, cands, mode, **kw):
    codes = O.encode(ps.ascii)
    params = P.Params(matrix=MAT, mode=mode, **kw)
    cells = torch.zeros(1, dtype=torch.int64, device="cuda")
    got = P.to_records(P.align_pairs(ctx, dev(codes), dev(ps.offsets), dev(cands.view(np.uint8).reshape(-1, 20)),
                                     params, cells), P.ALN_DTYPE)
    want, wcells = O.align_pairs(codes, ps.offsets, cands, MAT, params.gap_open, params.gap_extend, mode,
                                 params.xdrop, params.k, params.ani_min_pct, params.cov_min_pct)
    return got, want, int(cells.item()), wcells


def _cmp_alns(got, want):
    for f in ("score", "qb", "qe", "tb", "te", "ident", "cols", "seed_used", "passes"):
        bad = np.flatnonzero(got[f] != want[f])
        assert bad.size == 0, f"{f} differs at {bad[:5]}: {got[bad[:3]]} vs {want[bad[:3]]}"


@pytest.mark.parametrize("mode", [0, 1])
def test_align_parity_families(P, ctx, mode):
    ps = synth.families_1k()
    _, cands = _cands(P, ctx, ps)
    got, want, cells, wcells = _align_both(P, ctx, ps, cands, mode)
    _cmp_alns(got, want)
    assert cells == wcells


def _all_pairs(n):
    i, j = np.triu_indices(n, 1)
    c = np.zeros(i.size, O.CAND_DTYPE)
    c['i'], c['j'], c['count'] = i, j, 1
    return c


@pytest.mark.parametrize("o,e", [(11, 1), (3, 1), (1, 1), (64, 1), (65, 1), (0, 0), (20, 40)])
def test_sw_parity_edge_cases(P, ctx, o, e):
    ps = edge_case_set()
    cands = _all_pairs(ps.n)
    got, want, cells, wcells = _align_both(P, ctx, ps, cands, 0, gap_open=o, gap_extend=e)
    _cmp_alns(got, want)
    assert cells == wcells


def test_sw_parity_long_and_lopsided(P, ctx):
    rng = np.random.default_rng(3)
    fam = synth.planted_families([4, 3], 2, (1500, 2000), seed=5)
    short = synth.from_strings([''.join(rng.choice(list(synth.ALPHABET[:20]), size=L)) for L in (1, 31, 33, 257, 513)])
    strings = [fam.seq(i) for i in range(fam.n)] + [short.seq(i) for i in range(short.n)]
    ps = synth.from_strings(strings)
    cands = _all_pairs(ps.n)
    got, want, _, _ = _align_both(P, ctx, ps, cands, 0)
    _cmp_alns(got, want)


def test_sw_end_is_row_major_first_maximum(P, ctx):
    """Two cells share the best score (51): row 6 at column 44 and row 13 at column 4,
    both inside the first lane's block of rows.  The end must be the row-major first
    one, (6, 44), not the one met first column by column."""
    r = np.random.default_rng(4)

    def tf(n):
        return "".join(r.choice(list("ILV"), size=n))

    p1, p2 = "WCWCW", "CWCWW"
    t = p2 + tf(35) + p1 + tf(255)
    strings = [t]
    for tail in (488, 286, 120, 20):                 # 16, 10, 4 and 2 rows per lane
        strings.append("GG" + p1 + "GG" + p2 + "G" * tail)
    ps = synth.from_strings(strings)
    cands = _all_pairs(ps.n)
    got, want, _, _ = _align_both(P, ctx, ps, cands, 0)
    _cmp_alns(got, want)
    assert (got["score"][:ps.n - 1] == 51).all()
    swapped = synth.from_strings(strings[1:] + [t])
    cands = _all_pairs(swapped.n)
    got, want, _, _ = _align_both(P, ctx, swapped, cands, 0)
    _cmp_alns(got, want)
    last = want[cands["j"] == swapped.n - 1]         # (query, target): the query is the row
    assert (last["qe"] == 7).all() and (last["te"] == 45).all()


@pytest.mark.parametrize("X", [49, 5, 0, 1000])
def test_xd_parity_x_values(P, ctx, X):
    ps = synth.families_1k().subset(np.arange(300))
    _, cands = _cands(P, ctx, ps)
    got, want, cells, wcells = _align_both(P, ctx, ps, cands, 1, xdrop=X)
    _cmp_alns(got, want)
    assert cells == wcells


def test_xd_parity_substitute_seeds(P, ctx):
    ps = synth.zipf_100k(n=2000).subset(np.arange(200))
    _, cands = _cands(P, ctx, ps, m=25)
    got, want, cells, wcells = _align_both(P, ctx, ps, cands, 1)
    _cmp_alns(got, want)
    assert cells == wcells


def test_align_rejects_bad_pairs(P, ctx):
    ps = synth.families_1k().subset(np.arange(10))
    cands = _all_pairs(ps.n)
    cands['j'][3] = 10
    with pytest.raises(P.PastisError) as e:
        _align_both(P, ctx, ps, cands, 0)
    assert e.value.status == 1


def test_filter_and_end_to_end(P, ctx):
    ps = synth.families_1k()
    params = P.Params(matrix=MAT)
    res = P.run(ctx, dev(ps.ascii), dev(ps.offsets), params)
    ref = O.run(ps.ascii, ps.offsets, MAT)
    assert P.to_records(res["cands"], P.CAND_DTYPE).tobytes() == ref["cands"].tobytes()
    _cmp_alns(P.to_records(res["alns"], P.ALN_DTYPE), ref["alns"])
    assert P.to_records(res["edges"], P.EDGE_DTYPE).tobytes() == ref["edges"].tobytes()


def test_profiler_counts_kernels(P, ctx):
    ps = synth.families_1k().subset(np.arange(200))
    params = P.Params(matrix=MAT)
    for it in range(2):
        ctx.profile(True)
        r = P.run(ctx, dev(ps.ascii), dev(ps.offsets), params)
        prof = ctx.profile_read()
        st = ctx.stats()
        ctx.profile(False)
        for name in ("encode", "kmer_windows", "radix_scatter", "spgemm_cursors", "spgemm_rows", "sw_pass1", "sw_pass3",
                     "filter_flags"):
            assert name in prof and prof[name][0] >= 1 and prof[name][1] >= 0.0, name
        if it == 0:
            # the overlap product's work counters: one record per candidate, and at least
            # one product (posting entry) behind each unit of a record's count
            assert st["spgemm_records"] == r["cands"].shape[0]
            assert st["spgemm_products"] >= int(P.to_records(r["cands"], P.CAND_DTYPE)["count"].sum())
            # each left-operand entry once: the entries of the rows of A (exact k-mers,
            # every row but the last forms products over j > i)
            row_ptr, _, _ = O.kmers(O.encode(ps.ascii), ps.offsets, 6)
            assert st["spgemm_left_entries"] == int(row_ptr[-2])
            # the sorts that build A: every residue's window by code (24^6 codes: four
            # 8-bit passes), then the distinct k-mers by sequence (200 sequences: one)
            assert st["sort_element_passes"] == 4 * int(ps.offsets[-1]) + int(row_ptr[-1])


def test_spgemm_row_blocks_concatenate(P, ctx):
    ps = synth.zipf_100k(n=2000).subset(np.arange(400))
    codes = O.encode(ps.ascii)
    A = P.build_kmers(ctx, dev(codes), dev(ps.offsets), 6)
    params = P.Params(matrix=MAT, m_subs=25)
    whole = P.to_records(P.overlap_spgemm(ctx, A, params), P.CAND_DTYPE)
    parts = [P.to_records(P.overlap_spgemm(ctx, A, params, rows=(a, b)), P.CAND_DTYPE)
             for a, b in ((0, 37), (37, 37), (37, 250), (250, 400))]
    assert np.concatenate(parts).tobytes() == whole.tobytes()


def test_kept_as_reused_only_for_the_same_rows(P, ctx):
    """The AS matrix kept between row blocks gives the oracle's candidates in every block;
    A rebuilt in the same buffers with other rows (same size and entry count) is not
    mistaken for the kept one; pastis_ctx_forget makes the next call rebuild."""
    ps = synth.zipf_100k(n=2000).subset(np.arange(300))
    params = P.Params(matrix=MAT, m_subs=10)
    A = P.build_kmers(ctx, dev(O.encode(ps.ascii)), dev(ps.offsets), 6)

    def oracle_rows(s, a, b):
        rp, code, pos = O.kmers(O.encode(s.ascii), s.offsets, 6)
        c = O.candidates(rp, code, pos, 6, params.m_subs, MAT, 1)
        return c[(c['i'] >= a) & (c['i'] < b)]

    blocks = [(0, 60), (60, 150), (150, 300)]
    for a, b in blocks:                       # the first call builds AS, the others reuse it
        got = P.to_records(P.overlap_spgemm(ctx, A, params, rows=(a, b)), P.CAND_DTYPE)
        assert got.tobytes() == oracle_rows(ps, a, b).tobytes()
    # the first two sequences swapped: n and nnz(A) unchanged, the rows differ
    perm = np.arange(ps.n)
    perm[[0, 1]] = [1, 0]
    ps2 = ps.subset(perm)
    P.build_kmers(ctx, dev(O.encode(ps2.ascii)), dev(ps2.offsets), 6, A=A)
    got = P.to_records(P.overlap_spgemm(ctx, A, params, rows=(0, 60)), P.CAND_DTYPE)
    assert got.tobytes() == oracle_rows(ps2, 0, 60).tobytes()
    ctx.forget()
    again = P.to_records(P.overlap_spgemm(ctx, A, params, rows=(0, 60)), P.CAND_DTYPE)
    assert again.tobytes() == got.tobytes()



@pytest.mark.parametrize("which", ["families", "substitutes", "edge_cases"])
def test_align_filtered_parity(P, ctx, which):
    """PASTIS_SW_FILTERED against the oracle's mode 3: every field of every record, on
    family pairs (most pass), substitute-k-mer candidates (mostly random pairs, most cut
    before the traceback) and the edge-case set; and the same edges as PASTIS_SW."""
    if which == "families":
        ps = synth.families_1k()
        cands = _cands(P, ctx, ps)[1]
    elif which == "substitutes":
        ps = synth.zipf_100k(n=2000).subset(np.arange(300))
        cands = _cands(P, ctx, ps, m=25)[1]
    else:
        ps = edge_case_set()
        cands = _all_pairs(ps.n)
    got, want, gc, wc = _align_both(P, ctx, ps, cands, P.SW_FILTERED)
    assert gc == wc
    _cmp_alns(got, want)
    sw, _, _, _ = _align_both(P, ctx, ps, cands, P.SW)
    assert O.filter_edges(ps.offsets, cands, got).tobytes() == O.filter_edges(ps.offsets, cands, sw).tobytes()


@pytest.mark.parametrize("X", [0, 5, 49, 1000])
def test_xd_filtered_parity(P, ctx, X):
    """PASTIS_XD_FILTERED (extensions without carried statistics first, then again with
    them for the seeds that cover enough) against the oracle's mode 4, every field; the
    edges equal those of PASTIS_XD."""
    ps = synth.families_1k()
    cands = _cands(P, ctx, ps)[1]
    got, want, gc, wc = _align_both(P, ctx, ps, cands, P.XD_FILTERED, xdrop=X)
    assert gc == wc
    _cmp_alns(got, want)
    xd, _, _, _ = _align_both(P, ctx, ps, cands, P.XD, xdrop=X)
    assert O.filter_edges(ps.offsets, cands, got).tobytes() == O.filter_edges(ps.offsets, cands, xd).tobytes()


def test_xd_filtered_substitute_seeds(P, ctx):
    ps = synth.zipf_100k(n=2000).subset(np.arange(300))
    cands = _cands(P, ctx, ps, m=25)[1]
    got, want, gc, wc = _align_both(P, ctx, ps, cands, P.XD_FILTERED)
    assert gc == wc
    _cmp_alns(got, want)


def _xd_mat(scale):
    m = MAT.astype(np.int32) * scale
    return np.clip(m, -64, 63).astype(np.int8)


@pytest.mark.parametrize("per_warp", [0, 1, 2, 4])
@pytest.mark.parametrize("which", ["families", "wide", "edge_cases", "big_scores"])
def test_xd_lanes_parity(P, ctx, per_warp, which):
    """The x-drop in 16-bit lanes (1, 2 or 4 extensions per warp) or in 32-bit lanes,
    both modes: the filter-only mode (its first phase without carried statistics, its
    second with them) and the mode that carries them for every extension; every field
    against the oracle's.  'wide' (X = 1000) grows computed antidiagonals past the
    16-bit window, 'edge_cases' has seeds at sequence ends (sides of length 0) and short
    sequences, 'big_scores' a matrix whose scores times the extension length pass the
    16-bit bound: those extensions run in 32-bit lanes, with identical results."""
    mat, kw = MAT, {}
    if which == "edge_cases":
        ps = edge_case_set()
        cands = _cands(P, ctx, ps, k=2)[1]
        kw["k"] = 2
    elif which == "big_scores":
        ps = synth.families_1k().subset(np.arange(300))
        cands = _cands(P, ctx, ps)[1]
        mat = _xd_mat(6)
    else:
        ps = synth.families_1k()
        cands = _cands(P, ctx, ps)[1]
        if which == "wide":
            kw["xdrop"] = 1000
    assert len(cands) > 0
    codes = O.encode(ps.ascii)
    for mode in (P.XD_FILTERED, P.XD):
        params = P.Params(matrix=mat, mode=mode, **kw)
        ctx.set_xd_layout(per_warp)
        try:
            cells = torch.zeros(1, dtype=torch.int64, device="cuda")
            got = P.to_records(P.align_pairs(ctx, dev(codes), dev(ps.offsets),
                                             dev(cands.view(np.uint8).reshape(-1, 20)), params, cells), P.ALN_DTYPE)
        finally:
            ctx.set_xd_layout()
        want, wcells = O.align_pairs(codes, ps.offsets, cands, mat, params.gap_open, params.gap_extend, mode,
                                     params.xdrop, params.k, params.ani_min_pct, params.cov_min_pct)
        _cmp_alns(got, want)
        assert int(cells.item()) == wcells


@pytest.mark.parametrize("o,e,X", [(128, 1, 49), (129, 1, 49), (11, 1, 30000), (11, 1, 30001), (3, 1, 49),
                                   (1, 1, 5), (40, 30, 49)])
def test_xd_lanes_bounds(P, ctx, o, e, X):
    """At and past the 16-bit kernel's bounds (gap open or extend 128 vs 129, X 30,000 vs
    30,001) and with cheap or costly gaps (wide or narrow bands), every field of both
    x-drop modes equals the oracle's, in 16-bit lanes (four per warp) and in 32-bit
    lanes."""
    ps = synth.families_1k().subset(np.arange(400))
    cands = _cands(P, ctx, ps)[1]
    codes = O.encode(ps.ascii)
    for mode in (P.XD_FILTERED, P.XD):
        params = P.Params(matrix=MAT, mode=mode, gap_open=o, gap_extend=e, xdrop=X)
        want, wcells = O.align_pairs(codes, ps.offsets, cands, MAT, o, e, mode, X, params.k,
                                     params.ani_min_pct, params.cov_min_pct)
        for pw in (4, 0):
            ctx.set_xd_layout(pw)
            try:
                cells = torch.zeros(1, dtype=torch.int64, device="cuda")
                got = P.to_records(P.align_pairs(ctx, dev(codes), dev(ps.offsets),
                                                 dev(cands.view(np.uint8).reshape(-1, 20)), params, cells),
                                   P.ALN_DTYPE)
            finally:
                ctx.set_xd_layout()
            _cmp_alns(got, want)
            assert int(cells.item()) == wcells


def test_xd_layout_setting(P, ctx):
    assert ctx.xd_layout() == P.XD_DEFAULT_PER_WARP
    for bad in (-1, 3, 5, 8, 32):
        with pytest.raises(RuntimeError):
            ctx.set_xd_layout(bad)
        assert ctx.xd_layout() == P.XD_DEFAULT_PER_WARP
    for ok in (0, 1, 2, 4):
        ctx.set_xd_layout(ok)
        assert ctx.xd_layout() == ok
    ctx.set_xd_layout()
