/*
 * CPU oracle for the PASTIS hot path (Selvitopi et al., SC20, arXiv 2009.14467).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded C that states what the
 * path computes, step by step, for the parity tests, the smoke check and the CPU
 * baseline leg of the benchmark.  Nothing in the product path may call it.  It shares
 * no code, header, table or helper with the CUDA library: its record layouts are
 * declared here and mirrored by oracle/oracle.py alone.
 *
 * Steps (each function cites the passage it follows):
 *   or_encode          residue letters -> codes 0..23            Sec. V-B
 *   or_kmers           rows of A: (k-mer code, start position)   Sec. IV-A, Sec. V-B
 *   or_subkmers        m nearest substitute k-mers (rows of S)   Sec. IV-B, Alg. 1-3
 *   or_candidates      B = A A^T or A S A^T with the semiring     Sec. IV-A, IV-C
 *   or_sw              Smith-Waterman, affine gaps                Sec. IV-E, Sec. VI
 *   or_xd              x-drop seed-and-extend                     Sec. IV-E, Sec. VI
 *   or_align_pairs     SW or XD over a candidate list             Sec. IV-E
 *   or_filter          ANI / coverage similarity filter -> edges  Sec. IV-F, VI-B
 *   or_ns_edges        edges weighted by the normalized score     Sec. VI-B (NS)
 *   or_components      connected components of the edge graph    Sec. VI-B (components)
 *
 * Readings where the paper is silent are stated beside the code that takes them.
 * Two of them are definitions the paper does not give at all: the pruning order inside
 * or_xd (the paper hands x-drop to SeqAn) and the symmetrization rule inside
 * or_candidates.  The tests pin both to the reading stated here with cases worked out
 * by hand (every antidiagonal of small gapped extensions, the seed choice in each of its
 * branches, both orientations of a substitute pair) and with brute force; everything else
 * is pinned against brute force, closed forms and the values the paper prints.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NSYM 24
#define NEG (-1000000000)

/* ---- records (layout mirrored in oracle.py) ---------------------------- */
typedef struct {
    int32_t i, j;
    uint32_t count;
    uint16_t qpos[2];   /* seed start in sequence i (two smallest shared codes) */
    uint16_t tpos[2];   /* seed start in sequence j; 0xFFFF when absent         */
} or_cand;

typedef struct {
    int32_t score;
    uint16_t qb, qe, tb, te;  /* half-open spans [qb, qe) on i, [tb, te) on j */
    uint16_t ident, cols;
    uint8_t seed_used, passes;
    uint16_t pad;
} or_aln;

typedef struct {
    int32_t i, j;
    uint16_t ident, cols;
    int32_t score;
    float weight;
} or_edge;

/* ---- small growable arrays -------------------------------------------- */
typedef struct { void *p; int64_t n, cap; size_t elt; } vec;
static void vinit(vec *v, size_t elt) { v->p = NULL; v->n = 0; v->cap = 0; v->elt = elt; }
static void *vpush(vec *v) {
    if (v->n == v->cap) {
        int64_t nc = v->cap ? v->cap * 2 : 1024;
        void *np = realloc(v->p, (size_t)nc * v->elt);
        if (!np) return NULL;
        v->p = np; v->cap = nc;
    }
    return (char *)v->p + (size_t)(v->n++) * v->elt;
}

void or_free(void *p) { free(p); }

/* ======================================================================== */
/* Sec. V-B: the alphabet ARNDCQEGHILKMFPSTWYVBZX*, index 0..23.  Letters outside */
/* it (lower case included) are rejected (reading: the paper does not say).  */
/* Returns -1 when every byte is valid, else the index of the first bad one.  */
int64_t or_encode(const uint8_t *ascii, int64_t n, uint8_t *codes) {
    static const char alpha[] = "ARNDCQEGHILKMFPSTWYVBZX*";
    for (int64_t x = 0; x < n; ++x) {
        int c = -1;
        for (int a = 0; a < NSYM; ++a)
            if ((uint8_t)alpha[a] == ascii[x]) { c = a; break; }
        if (c < 0) return x;
        codes[x] = (uint8_t)c;
    }
    return -1;
}

/* ======================================================================== */
/* Sec. V-B: id = sum_t c(s[p+t]) * 24^(k-1-t) (the leftmost letter is the most */
/* significant).  Sec. IV-A: A_ij holds the start position of k-mer j in       */
/* sequence i.  Reading: positions are 0-based, and a k-mer repeated in one    */
/* sequence keeps its smallest start position (one value per matrix cell).     */
static uint32_t kmer_code(const uint8_t *s, int k) {
    uint32_t c = 0;
    for (int t = 0; t < k; ++t) c = c * NSYM + s[t];
    return c;
}

typedef struct { uint32_t code; uint32_t pos; } code_pos;
static int cmp_code_pos(const void *a, const void *b) {
    const code_pos *x = a, *y = b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

/* Rows of A for all sequences: row_ptr[n+1], codes ascending within a row.   */
int64_t or_kmers(const uint8_t *codes, const int64_t *offsets, int32_t n, int32_t k,
                 int64_t *row_ptr, uint32_t *out_code, uint16_t *out_pos) {
    int64_t nnz = 0;
    row_ptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t L = offsets[i + 1] - offsets[i];
        const uint8_t *s = codes + offsets[i];
        if (L >= k) {
            int64_t cnt = L - k + 1;
            code_pos *tmp = malloc(sizeof(code_pos) * (size_t)cnt);
            for (int64_t p = 0; p < cnt; ++p) { tmp[p].code = kmer_code(s + p, k); tmp[p].pos = (uint32_t)p; }
            qsort(tmp, (size_t)cnt, sizeof(code_pos), cmp_code_pos);
            for (int64_t p = 0; p < cnt; ++p) {
                if (p > 0 && tmp[p].code == tmp[p - 1].code) continue;
                out_code[nnz] = tmp[p].code;
                out_pos[nnz] = (uint16_t)tmp[p].pos;
                ++nnz;
            }
            free(tmp);
        }
        row_ptr[i + 1] = nnz;
    }
    return nnz;
}

/* ======================================================================== */
/* Sec. IV-B.  Expense of replacing base a by b: C[a][a] - C[a][b] (the matrix   */
/* E = Sort(Diag(C) - C)).  The distance of k-mer q from root r is the sum of    */
/* the expenses over positions; it is not symmetric.  N_m(r) is the set of the   */
/* m k-mers q != r nearest to r (ties: smaller code first, a reading: Alg. 1-3   */
/* do not order equal distances).  This oracle computes that set by its plain    */
/* definition instead of the best-first search of Alg. 1-3: count the k-mers     */
/* within distance D by depth-first enumeration, raise D until at least m are    */
/* found, then sort them by (distance, code) and keep m.  Row r of S lists the   */
/* identity (r, 0) first (reading: without it A S A^T would lose exact matches), */
/* then N_m(r).  Substitutes range over all 24 symbols.                         */
typedef struct { int32_t dist; uint32_t code; } sub_ent;
static int cmp_sub(const void *a, const void *b) {
    const sub_ent *x = a, *y = b;
    if (x->dist != y->dist) return x->dist < y->dist ? -1 : 1;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    return 0;
}

typedef struct {
    int k;
    const uint8_t *root;
    int32_t exp_[NSYM][NSYM];     /* expense a -> b */
    int32_t suffix_min[8];        /* least expense obtainable from position t on */
    int32_t D;
    vec *out;                      /* sub_ent, collected when out != NULL */
    int64_t count;
} dfs_ctx;

static void dfs(dfs_ctx *c, int t, uint32_t code, int32_t dist, int changed) {
    if (dist + c->suffix_min[t] > c->D) return;
    if (t == c->k) {
        if (!changed) return;               /* q != r */
        c->count++;
        if (c->out) { sub_ent *e = vpush(c->out); e->dist = dist; e->code = code; }
        return;
    }
    int a = c->root[t];
    for (int b = 0; b < NSYM; ++b)
        dfs(c, t + 1, code * NSYM + (uint32_t)b, dist + c->exp_[a][b], changed || b != a);
}

int or_subkmers(const uint32_t *roots, int64_t n_roots, int32_t k, int32_t m,
                const int8_t *matrix, uint32_t *out_code, int32_t *out_dist) {
    if (k < 1 || k > 6 || m < 0) return -1;
    int64_t space = 1;
    for (int t = 0; t < k; ++t) space *= NSYM;
    if (m > space - 1) return -1;
    dfs_ctx c;
    c.k = k;
    for (int a = 0; a < NSYM; ++a)
        for (int b = 0; b < NSYM; ++b)
            c.exp_[a][b] = (int32_t)matrix[a * NSYM + a] - (int32_t)matrix[a * NSYM + b];
    uint8_t root[8];
    c.root = root;
    for (int64_t r = 0; r < n_roots; ++r) {
        uint32_t x = roots[r];
        for (int t = k - 1; t >= 0; --t) { root[t] = (uint8_t)(x % NSYM); x /= NSYM; }
        c.suffix_min[k] = 0;
        int32_t lo = 0;
        for (int t = k - 1; t >= 0; --t) {
            int32_t mn = c.exp_[root[t]][0];
            for (int b = 1; b < NSYM; ++b) if (c.exp_[root[t]][b] < mn) mn = c.exp_[root[t]][b];
            c.suffix_min[t] = c.suffix_min[t + 1] + mn;
        }
        lo = c.suffix_min[0];
        out_code[r * (m + 1)] = roots[r];
        out_dist[r * (m + 1)] = 0;
        if (m == 0) continue;
        c.out = NULL;
        int32_t D = lo;
        for (;;) {
            c.D = D; c.count = 0;
            dfs(&c, 0, 0, 0, 0);
            if (c.count >= m) break;
            ++D;
        }
        vec v; vinit(&v, sizeof(sub_ent));
        c.out = &v; c.D = D; c.count = 0;
        dfs(&c, 0, 0, 0, 0);
        qsort(v.p, (size_t)v.n, sizeof(sub_ent), cmp_sub);
        sub_ent *e = v.p;
        for (int t = 0; t < m; ++t) {
            out_code[r * (m + 1) + 1 + t] = e[t].code;
            out_dist[r * (m + 1) + 1 + t] = e[t].dist;
        }
        free(v.p);
    }
    return 0;
}

/* ======================================================================== */
/* Candidate pairs.  Sec. IV-A: B = A A^T under a semiring whose multiply pairs */
/* the two start positions of a shared k-mer and whose add counts the shared    */
/* k-mers and keeps at most two seeds; B is symmetric, so only i < j is kept.    */
/* Reading: the two seeds are the two shared k-mers with the smallest codes.    */
/* Sec. IV-C: with substitutes the product is (A S) A^T, where AS(i, s) is the  */
/* start of the k-mer of i closest to s (ties: smaller start, reading of the     */
/* "<=" in Sec. IV-C), and the result is symmetrized (Sec. VI-A dissection).     */
/* Reading for symmetrization: for i < j take the orientation with more shared  */
/* substitutes, (i, j) on a tie; seeds are reported as (pos in i, pos in j).    */
/* Sec. VI: pairs sharing fewer than min_shared k-mers are dropped.             */
typedef struct { uint32_t code; int32_t seq; uint32_t pos; int32_t dist; } posting;
static int cmp_posting(const void *a, const void *b) {
    const posting *x = a, *y = b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    if (x->seq != y->seq) return x->seq < y->seq ? -1 : 1;
    if (x->dist != y->dist) return x->dist < y->dist ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

typedef struct { int32_t i, j; uint32_t code; uint16_t pi, pj; } product;
static int cmp_product(const void *a, const void *b) {
    const product *x = a, *y = b;
    if (x->i != y->i) return x->i < y->i ? -1 : 1;
    if (x->j != y->j) return x->j < y->j ? -1 : 1;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    return 0;
}

typedef struct { int32_t i, j; uint32_t count; uint32_t code[2]; uint16_t pi[2], pj[2]; } ordered;

static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y);
}

/* Reduce sorted products into one record per ordered pair. */
static ordered *reduce_products(product *pr, int64_t np, int64_t *n_out) {
    ordered *o = malloc(sizeof(ordered) * (size_t)(np ? np : 1));
    int64_t no = 0;
    for (int64_t x = 0; x < np;) {
        int64_t y = x;
        while (y < np && pr[y].i == pr[x].i && pr[y].j == pr[x].j) ++y;
        ordered *r = &o[no++];
        r->i = pr[x].i; r->j = pr[x].j; r->count = (uint32_t)(y - x);
        for (int t = 0; t < 2; ++t) {
            if (x + t < y) { r->code[t] = pr[x + t].code; r->pi[t] = pr[x + t].pi; r->pj[t] = pr[x + t].pj; }
            else { r->code[t] = 0xFFFFFFFFu; r->pi[t] = 0xFFFF; r->pj[t] = 0xFFFF; }
        }
        x = y;
    }
    *n_out = no;
    return o;
}

static int64_t find_ordered(const ordered *o, int64_t n, int32_t i, int32_t j) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (o[mid].i < i || (o[mid].i == i && o[mid].j < j)) lo = mid + 1; else hi = mid;
    }
    return (lo < n && o[lo].i == i && o[lo].j == j) ? lo : -1;
}

static int cmp_cand(const void *a, const void *b) {
    const or_cand *x = a, *y = b;
    if (x->i != y->i) return x->i < y->i ? -1 : 1;
    if (x->j != y->j) return x->j < y->j ? -1 : 1;
    return 0;
}

int or_candidates(const int64_t *row_ptr, const uint32_t *code, const uint16_t *pos, int32_t n,
                  int32_t k, int32_t m, const int8_t *matrix, int32_t min_shared,
                  or_cand **out, int64_t *n_out) {
    int64_t nnz = row_ptr[n];
    /* postings of A: (code, seq, pos) */
    posting *pa = malloc(sizeof(posting) * (size_t)(nnz ? nnz : 1));
    for (int32_t i = 0; i < n; ++i)
        for (int64_t x = row_ptr[i]; x < row_ptr[i + 1]; ++x) {
            pa[x].code = code[x]; pa[x].seq = i; pa[x].pos = pos[x]; pa[x].dist = 0;
        }
    qsort(pa, (size_t)nnz, sizeof(posting), cmp_posting);

    vec prods; vinit(&prods, sizeof(product));
    if (m == 0) {
        /* exact: every pair of postings of one code, i < j */
        for (int64_t x = 0; x < nnz;) {
            int64_t y = x;
            while (y < nnz && pa[y].code == pa[x].code) ++y;
            for (int64_t a = x; a < y; ++a)
                for (int64_t b = a + 1; b < y; ++b) {
                    product *p = vpush(&prods);
                    p->i = pa[a].seq; p->j = pa[b].seq; p->code = pa[a].code;
                    p->pi = (uint16_t)pa[a].pos; p->pj = (uint16_t)pa[b].pos;
                }
            x = y;
        }
    } else {
        /* S for every distinct k-mer present */
        uint32_t *roots = malloc(sizeof(uint32_t) * (size_t)(nnz ? nnz : 1));
        int64_t nr = 0;
        for (int64_t x = 0; x < nnz; ++x)
            if (x == 0 || pa[x].code != pa[x - 1].code) roots[nr++] = pa[x].code;
        uint32_t *sc = malloc(sizeof(uint32_t) * (size_t)(nr ? nr : 1) * (size_t)(m + 1));
        int32_t *sd = malloc(sizeof(int32_t) * (size_t)(nr ? nr : 1) * (size_t)(m + 1));
        if (or_subkmers(roots, nr, k, m, matrix, sc, sd) != 0) return -1;
        /* AS: for each (i, s) the start of the k-mer of i closest to s */
        vec as; vinit(&as, sizeof(posting));
        for (int32_t i = 0; i < n; ++i)
            for (int64_t x = row_ptr[i]; x < row_ptr[i + 1]; ++x) {
                uint32_t *hit = bsearch(&code[x], roots, (size_t)nr, sizeof(uint32_t), cmp_u32);
                int64_t r = hit - roots;
                for (int t = 0; t <= m; ++t) {
                    posting *p = vpush(&as);
                    p->code = sc[r * (m + 1) + t]; p->seq = i; p->pos = pos[x];
                    p->dist = sd[r * (m + 1) + t];
                }
            }
        qsort(as.p, (size_t)as.n, sizeof(posting), cmp_posting);
        posting *ap = as.p;
        int64_t nas = 0;   /* keep the first (smallest dist, then pos) per (code, seq) */
        for (int64_t x = 0; x < as.n; ++x)
            if (nas == 0 || ap[x].code != ap[nas - 1].code || ap[x].seq != ap[nas - 1].seq)
                ap[nas++] = ap[x];
        /* (AS) A^T: each substitute s of i that is a k-mer of j, ordered pairs i != j */
        int64_t y = 0;
        for (int64_t x = 0; x < nas;) {
            int64_t x2 = x;
            while (x2 < nas && ap[x2].code == ap[x].code) ++x2;
            while (y < nnz && pa[y].code < ap[x].code) ++y;
            int64_t y2 = y;
            while (y2 < nnz && pa[y2].code == ap[x].code) ++y2;
            for (int64_t a = x; a < x2; ++a)
                for (int64_t b = y; b < y2; ++b) {
                    if (ap[a].seq == pa[b].seq) continue;
                    product *p = vpush(&prods);
                    p->i = ap[a].seq; p->j = pa[b].seq; p->code = ap[a].code;
                    p->pi = (uint16_t)ap[a].pos; p->pj = (uint16_t)pa[b].pos;
                }
            x = x2;
        }
        free(as.p); free(roots); free(sc); free(sd);
    }
    free(pa);
    qsort(prods.p, (size_t)prods.n, sizeof(product), cmp_product);
    int64_t no;
    ordered *o = reduce_products(prods.p, prods.n, &no);
    free(prods.p);

    or_cand *res = malloc(sizeof(or_cand) * (size_t)(no ? no : 1));
    int64_t nc = 0;
    for (int64_t x = 0; x < no; ++x) {
        const ordered *f = &o[x], *use = f;
        int swap = 0;
        if (m == 0) {
            /* products were built with i < j already */
        } else {
            if (f->i < f->j) {
                int64_t b = find_ordered(o, no, f->j, f->i);
                if (b >= 0 && o[b].count > f->count) { use = &o[b]; swap = 1; }
            } else {
                /* (i, j) with i > j: emitted here only when (j, i) has no record */
                if (find_ordered(o, no, f->j, f->i) >= 0) continue;
                swap = 1;
            }
        }
        if (use->count < (uint32_t)min_shared) continue;
        or_cand *c = &res[nc++];
        c->count = use->count;
        if (!swap) {
            c->i = use->i; c->j = use->j;
            for (int t = 0; t < 2; ++t) { c->qpos[t] = use->pi[t]; c->tpos[t] = use->pj[t]; }
        } else {
            c->i = use->j; c->j = use->i;
            for (int t = 0; t < 2; ++t) { c->qpos[t] = use->pj[t]; c->tpos[t] = use->pi[t]; }
        }
    }
    free(o);
    qsort(res, (size_t)nc, sizeof(or_cand), cmp_cand);
    *out = res;
    *n_out = nc;
    return 0;
}

/* ======================================================================== */
/* Sec. IV-E, Sec. VI: Smith-Waterman local alignment, BLOSUM62, gap open 11,   */
/* extension 1.  Reading of the gap cost: a gap of length L costs               */
/* open + (L-1)*extend.  Textbook Gotoh recurrences over the full matrices:     */
/*   E(i,j) = max(H(i,j-1) - o, E(i,j-1) - e)        (gap in q, moves along j)  */
/*   F(i,j) = max(H(i-1,j) - o, F(i-1,j) - e)        (gap in t, moves along i)  */
/*   H(i,j) = max(0, H(i-1,j-1) + s(q_i,t_j), F(i,j), E(i,j))                   */
/* The end cell is the first maximum in row-major order.  The alignment is then */
/* traced back from it with these priorities (a reading; they fix one optimal   */
/* alignment): in H prefer the diagonal, then F, then E; in E and F prefer the  */
/* gap open over the extension; stop at a diagonal step whose predecessor H is  */
/* 0.  ident counts columns with equal residues, cols counts every column.      */
typedef struct { int32_t score; int32_t qb, qe, tb, te, ident, cols; } span_stats;

static int32_t sub_score(const int8_t *mat, uint8_t a, uint8_t b) { return mat[a * NSYM + b]; }

void or_sw(const uint8_t *q, int32_t lq, const uint8_t *t, int32_t lt, const int8_t *mat,
           int32_t o, int32_t e, span_stats *res) {
    int64_t W = lt + 1;
    int32_t *H = malloc(sizeof(int32_t) * (size_t)(lq + 1) * (size_t)W);
    int32_t *E = malloc(sizeof(int32_t) * (size_t)(lq + 1) * (size_t)W);
    int32_t *F = malloc(sizeof(int32_t) * (size_t)(lq + 1) * (size_t)W);
#define AT(M, i, j) M[(int64_t)((i) + 1) * W + ((j) + 1)]
    for (int32_t j = -1; j < lt; ++j) { AT(H, -1, j) = 0; AT(E, -1, j) = NEG; AT(F, -1, j) = NEG; }
    for (int32_t i = 0; i < lq; ++i) { AT(H, i, -1) = 0; AT(E, i, -1) = NEG; AT(F, i, -1) = NEG; }
    int32_t best = 0, bi = -1, bj = -1;
    for (int32_t i = 0; i < lq; ++i)
        for (int32_t j = 0; j < lt; ++j) {
            int32_t ev = AT(H, i, j - 1) - o, ex = AT(E, i, j - 1) - e;
            int32_t Ev = ev > ex ? ev : ex; if (Ev < NEG) Ev = NEG;
            int32_t fv = AT(H, i - 1, j) - o, fx = AT(F, i - 1, j) - e;
            int32_t Fv = fv > fx ? fv : fx; if (Fv < NEG) Fv = NEG;
            int32_t D = AT(H, i - 1, j - 1) + sub_score(mat, q[i], t[j]);
            int32_t h = 0;
            if (D > h) h = D;
            if (Fv > h) h = Fv;
            if (Ev > h) h = Ev;
            AT(H, i, j) = h; AT(E, i, j) = Ev; AT(F, i, j) = Fv;
            if (h > best) { best = h; bi = i; bj = j; }
        }
    memset(res, 0, sizeof(*res));
    if (best > 0) {
        int32_t i = bi, j = bj, state = 0; /* 0 = H, 1 = F, 2 = E */
        int32_t ident = 0, cols = 0;
        for (;;) {
            if (state == 0) {
                int32_t h = AT(H, i, j);
                if (AT(H, i - 1, j - 1) + sub_score(mat, q[i], t[j]) == h) {
                    ++cols; ident += (q[i] == t[j]);
                    if (AT(H, i - 1, j - 1) == 0) break;
                    --i; --j;
                } else if (AT(F, i, j) == h) state = 1;
                else state = 2;
            } else if (state == 1) {
                ++cols;
                state = (AT(H, i - 1, j) - o >= AT(F, i - 1, j) - e) ? 0 : 1;
                --i;
            } else {
                ++cols;
                state = (AT(H, i, j - 1) - o >= AT(E, i, j - 1) - e) ? 0 : 2;
                --j;
            }
        }
        res->score = best;
        res->qb = i; res->qe = bi + 1; res->tb = j; res->te = bj + 1;
        res->ident = ident; res->cols = cols;
    }
#undef AT
    free(H); free(E); free(F);
}

/* ======================================================================== */
/* Sec. IV-E, Sec. VI: x-drop extension (X = 49), computed antidiagonal by       */
/* antidiagonal; the paper hands this to SeqAn and gives no algorithm, so this   */
/* is the reading the oracle fixes.  Cell (a, b) has consumed a residues of q'   */
/* and b of t'; (0,0) is the anchor with H = 0.  No zero clamp:                  */
/*   E(a,b) = max(H(a,b-1) - o, E(a,b-1) - e)    F(a,b) = max(H(a-1,b) - o, ...)  */
/*   H(a,b) = max(H(a-1,b-1) + s(q'_{a-1}, t'_{b-1}), F(a,b), E(a,b))           */
/* Antidiagonal d+1 is computed for a in [lo_d, hi_d + 1] (clipped to the        */
/* matrix), where [lo_d, hi_d] are the first and last live cells of d.  After    */
/* an antidiagonal is computed, its cells with H < best - X die (H = E = F =     */
/* -inf), where best is the maximum over the earlier antidiagonals; then best is */
/* raised by the live cells.  The extension stops when no cell stays live.  The  */
/* end is the first cell (antidiagonal, then a) reaching best; the path back to  */
/* the anchor follows the same priorities as or_sw.  `cells` counts computed     */
/* cells.                                                                        */
typedef struct { int32_t score, a, b, ident, cols; int64_t cells; } ext_res;

static void xd_extend(const uint8_t *q, int32_t A, int32_t qs, const uint8_t *t, int32_t B,
                      int32_t ts, const int8_t *mat, int32_t o, int32_t e, int32_t X,
                      ext_res *res) {
    int32_t ND = A + B + 1;
    int32_t *lo = malloc(sizeof(int32_t) * (size_t)ND), *hi = malloc(sizeof(int32_t) * (size_t)ND);
    int64_t *base = malloc(sizeof(int64_t) * (size_t)ND);
    vec Hv, Ev, Fv; vinit(&Hv, 4); vinit(&Ev, 4); vinit(&Fv, 4);
#define QC(a) q[(int64_t)(a) * qs]
#define TC(b) t[(int64_t)(b) * ts]
    /* value lookup on a stored antidiagonal; outside the computed range: -inf */
#define GET(V, d, a) (((d) >= 0 && (d) <= dmax && (a) >= lo[d] && (a) <= hi[d]) ? \
                      ((int32_t *)V.p)[base[d] + (a) - lo[d]] : NEG)
    int32_t dmax = 0;
    lo[0] = 0; hi[0] = 0; base[0] = 0;
    *(int32_t *)vpush(&Hv) = 0; *(int32_t *)vpush(&Ev) = NEG; *(int32_t *)vpush(&Fv) = NEG;
    int32_t best = 0, ba = 0, bb = 0;
    int64_t cells = 1;
    int32_t llo = 0, lhi = 0;               /* live range of the last antidiagonal */
    for (int32_t d = 1; d < ND; ++d) {
        int32_t clo = llo, chi = lhi + 1;
        if (clo < d - B) clo = d - B;
        if (chi > A) chi = A;
        if (clo < 0) clo = 0;
        if (chi > d) chi = d;
        if (clo > chi) break;
        lo[d] = clo; hi[d] = chi; base[d] = Hv.n; dmax = d;
        for (int32_t a = clo; a <= chi; ++a) {
            int32_t b = d - a;
            int32_t Evv = NEG, Fvv = NEG, Dv = NEG;
            if (b >= 1) {
                int32_t x1 = GET(Hv, d - 1, a) - o, x2 = GET(Ev, d - 1, a) - e;
                Evv = x1 > x2 ? x1 : x2; if (Evv < NEG) Evv = NEG;
            }
            if (a >= 1) {
                int32_t x1 = GET(Hv, d - 1, a - 1) - o, x2 = GET(Fv, d - 1, a - 1) - e;
                Fvv = x1 > x2 ? x1 : x2; if (Fvv < NEG) Fvv = NEG;
            }
            if (a >= 1 && b >= 1) {
                int32_t hd = GET(Hv, d - 2, a - 1);
                Dv = hd == NEG ? NEG : hd + sub_score(mat, QC(a - 1), TC(b - 1));
            }
            int32_t h = Dv;
            if (Fvv > h) h = Fvv;
            if (Evv > h) h = Evv;
            *(int32_t *)vpush(&Hv) = h; *(int32_t *)vpush(&Ev) = Evv; *(int32_t *)vpush(&Fv) = Fvv;
            ++cells;
        }
        int32_t nlo = -1, nhi = -1, dbest = NEG, dba = -1;
        for (int32_t a = clo; a <= chi; ++a) {
            int32_t *h = &((int32_t *)Hv.p)[base[d] + a - clo];
            if (*h < best - X) {
                *h = NEG;
                ((int32_t *)Ev.p)[base[d] + a - clo] = NEG;
                ((int32_t *)Fv.p)[base[d] + a - clo] = NEG;
                continue;
            }
            if (nlo < 0) nlo = a;
            nhi = a;
            if (*h > dbest) { dbest = *h; dba = a; }
        }
        if (nlo < 0) break;
        if (dbest > best) { best = dbest; ba = dba; bb = d - dba; }
        llo = nlo; lhi = nhi;
    }
    /* trace back from (ba, bb) to the anchor */
    int32_t a = ba, b = bb, state = 0, ident = 0, ncols = 0;
    while (!(state == 0 && a == 0 && b == 0)) {
        int32_t d = a + b;
        if (state == 0) {
            int32_t h = GET(Hv, d, a);
            int32_t hd = (a >= 1 && b >= 1) ? GET(Hv, d - 2, a - 1) : NEG;
            if (hd != NEG && hd + sub_score(mat, QC(a - 1), TC(b - 1)) == h) {
                ++ncols; ident += (QC(a - 1) == TC(b - 1)); --a; --b;
            } else if (GET(Fv, d, a) == h) state = 1;
            else state = 2;
        } else if (state == 1) {
            ++ncols;
            state = (GET(Hv, d - 1, a - 1) - o >= GET(Fv, d - 1, a - 1) - e) ? 0 : 1;
            --a;
        } else {
            ++ncols;
            state = (GET(Hv, d - 1, a) - o >= GET(Ev, d - 1, a) - e) ? 0 : 2;
            --b;
        }
    }
#undef GET
#undef QC
#undef TC
    res->score = best; res->a = ba; res->b = bb; res->ident = ident; res->cols = ncols;
    res->cells = cells;
    free(lo); free(hi); free(base); free(Hv.p); free(Ev.p); free(Fv.p);
}

/* Seed-and-extend from one seed (pi, pj): seed score + left + right extension. */
void or_xd(const uint8_t *q, int32_t lq, const uint8_t *t, int32_t lt, int32_t pi, int32_t pj,
           int32_t k, const int8_t *mat, int32_t o, int32_t e, int32_t X, span_stats *res,
           int64_t *cells) {
    int32_t seed = 0, sid = 0;
    for (int32_t x = 0; x < k; ++x) {
        seed += sub_score(mat, q[pi + x], t[pj + x]);
        sid += (q[pi + x] == t[pj + x]);
    }
    ext_res R, L;
    xd_extend(q + pi + k, lq - pi - k, 1, t + pj + k, lt - pj - k, 1, mat, o, e, X, &R);
    xd_extend(q + pi - 1, pi, -1, t + pj - 1, pj, -1, mat, o, e, X, &L);
    res->score = L.score + seed + R.score;
    res->qb = pi - L.a; res->tb = pj - L.b;
    res->qe = pi + k + R.a; res->te = pj + k + R.b;
    res->ident = L.ident + sid + R.ident;
    res->cols = L.cols + k + R.cols;
    if (cells) *cells += L.cells + R.cells;
}

/* ======================================================================== */
/* Sec. IV-F, Sec. VI-B: veto ANI < ani% or shorter-sequence coverage < cov%.  */
/* Readings: ANI = identical columns / all columns (gap columns included);      */
/* coverage = aligned span on the shorter sequence over its length (sequence i  */
/* on equal lengths); both tests are exact integer comparisons, inclusive.      */
static int passes(const span_stats *s, int32_t lq, int32_t lt, int32_t ani, int32_t cov) {
    if (s->cols <= 0) return 0;
    int32_t span = lq <= lt ? s->qe - s->qb : s->te - s->tb;
    int32_t L = lq <= lt ? lq : lt;
    return (int64_t)100 * s->ident >= (int64_t)ani * s->cols &&
           (int64_t)100 * span >= (int64_t)cov * L;
}

/* Sec. IV-E: SW ignores the seeds; XD extends from each of the (at most two)   */
/* seeds and keeps the best alignment that passes the filter.  Reading: among   */
/* passing seeds the higher score wins, the first seed on a tie; when none     */
/* passes, the best score is reported (first seed on a tie) with passes = 0.    */
/* Modes 3 and 4 are SW and XD for the filter of Sec. IV-F only: a pair that    */
/* fails keeps its score and end (and, for XD, the seed kept), and its begin,   */
/* identities and columns are reported as 0.                                    */
int or_align_pairs(const uint8_t *codes, const int64_t *offsets, const or_cand *pairs,
                   int64_t n_pairs, const int8_t *mat, int32_t o, int32_t e, int32_t mode,
                   int32_t X, int32_t k, int32_t ani, int32_t cov, or_aln *out, int64_t *cells) {
    for (int64_t p = 0; p < n_pairs; ++p) {
        const or_cand *c = &pairs[p];
        const uint8_t *q = codes + offsets[c->i], *t = codes + offsets[c->j];
        int32_t lq = (int32_t)(offsets[c->i + 1] - offsets[c->i]);
        int32_t lt = (int32_t)(offsets[c->j + 1] - offsets[c->j]);
        span_stats best;
        int used = 0, ok = 0;
        if (mode == 0 || mode == 2 || mode == 3) {
            or_sw(q, lq, t, lt, mat, o, e, &best);
            if (cells) *cells += (int64_t)lq * lt;
            ok = passes(&best, lq, lt, ani, cov);
            if (mode == 3 && !ok) {
                best.qb = best.tb = 0;
                best.ident = best.cols = 0;
            }
            if (mode == 2) {
                /* score and end only (what the NS weight needs, Sec. VI-B: no traceback) */
                best.qb = best.tb = 0;
                best.ident = best.cols = 0;
                ok = 0;
            }
        } else {
            int ns = (c->count >= 2 && c->qpos[1] != 0xFFFF) ? 2 : 1;
            for (int s = 0; s < ns; ++s) {
                span_stats cur;
                or_xd(q, lq, t, lt, c->qpos[s], c->tpos[s], k, mat, o, e, X, &cur, cells);
                int pc = passes(&cur, lq, lt, ani, cov);
                int take;
                if (s == 0) take = 1;
                else if (pc != ok) take = pc;          /* a passing seed beats a failing one */
                else take = cur.score > best.score;    /* same status: higher score */
                if (take) { best = cur; used = s; ok = pc; }
            }
            if (mode == 4 && !ok) {
                best.qb = best.tb = 0;
                best.ident = best.cols = 0;
            }
        }
        or_aln *r = &out[p];
        r->score = best.score;
        r->qb = (uint16_t)best.qb; r->qe = (uint16_t)best.qe;
        r->tb = (uint16_t)best.tb; r->te = (uint16_t)best.te;
        r->ident = (uint16_t)best.ident; r->cols = (uint16_t)best.cols;
        r->seed_used = (uint8_t)used; r->passes = (uint8_t)ok; r->pad = 0;
    }
    return 0;
}

/* NS edges (Sec. VI-B): the raw score normalized by the shorter sequence, which needs
 * no traceback.  Reading: weight = score / min(|s_i|, |s_j|) in float32; the ANI and
 * coverage tests need the traceback and do not apply, so every pair with a positive
 * score is an edge.  Input (i, j) order. */
int64_t or_ns_edges(const int64_t *offsets, const or_cand *pairs, const or_aln *alns, int64_t n_pairs,
                    or_edge *out) {
    int64_t ne = 0;
    for (int64_t p = 0; p < n_pairs; ++p) {
        if (alns[p].score <= 0) continue;
        int64_t lq = offsets[pairs[p].i + 1] - offsets[pairs[p].i];
        int64_t lt = offsets[pairs[p].j + 1] - offsets[pairs[p].j];
        int64_t ls = lq < lt ? lq : lt;
        or_edge *x = &out[ne++];
        x->i = pairs[p].i; x->j = pairs[p].j;
        x->ident = alns[p].ident; x->cols = alns[p].cols; x->score = alns[p].score;
        x->weight = (float)alns[p].score / (float)ls;
    }
    return ne;
}

/* Connected components of the graph on n vertices with the given edges (the paper's
 * components-as-families variant, Sec. VI-B).  label[v] = the smallest vertex of v's
 * component: union-find that always hangs the larger root under the smaller one. */
static int32_t uf_find(int32_t *parent, int32_t v) {
    while (parent[v] != v) {
        parent[v] = parent[parent[v]];
        v = parent[v];
    }
    return v;
}

int or_components(int32_t n, const or_edge *edges, int64_t n_edges, int32_t *label) {
    for (int32_t v = 0; v < n; ++v) label[v] = v;
    for (int64_t x = 0; x < n_edges; ++x) {
        int32_t a = edges[x].i, b = edges[x].j;
        if (a < 0 || b < 0 || a >= n || b >= n) return 1;
        a = uf_find(label, a);
        b = uf_find(label, b);
        if (a < b) label[b] = a;
        else if (b < a) label[a] = b;
    }
    for (int32_t v = 0; v < n; ++v) label[v] = uf_find(label, v);
    return 0;
}

/* Edges in input (i, j) order; weight = ANI = ident / cols (Sec. VI-B). */
int64_t or_filter(const int64_t *offsets, const or_cand *pairs, const or_aln *alns,
                  int64_t n_pairs, int32_t ani, int32_t cov, or_edge *out) {
    int64_t ne = 0;
    for (int64_t p = 0; p < n_pairs; ++p) {
        span_stats s;
        s.score = alns[p].score;
        s.qb = alns[p].qb; s.qe = alns[p].qe; s.tb = alns[p].tb; s.te = alns[p].te;
        s.ident = alns[p].ident; s.cols = alns[p].cols;
        int32_t lq = (int32_t)(offsets[pairs[p].i + 1] - offsets[pairs[p].i]);
        int32_t lt = (int32_t)(offsets[pairs[p].j + 1] - offsets[pairs[p].j]);
        if (!passes(&s, lq, lt, ani, cov)) continue;
        or_edge *x = &out[ne++];
        x->i = pairs[p].i; x->j = pairs[p].j;
        x->ident = (uint16_t)s.ident; x->cols = (uint16_t)s.cols; x->score = s.score;
        x->weight = (float)s.ident / (float)s.cols;
    }
    return ne;
}
