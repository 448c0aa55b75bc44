/*
 * pastis.h - C ABI of the GB300 (sm_103a) PASTIS hot path.
 *
 * PASTIS (Selvitopi, Ekanayake, Guidi, Pavlopoulos, Azad, Buluc; SC20, arXiv
 * 2009.14467) builds a protein similarity graph G = (V, E): V is the set of
 * sequences, and an edge joins two sequences whose alignment passes the similarity
 * thresholds (Sec. II).  The hot path this library runs on one GPU:
 *
 *   pastis_encode            letters -> residue codes                (Sec. V-B)
 *   pastis_build_kmers       A (sequence x k-mer) in CSR and CSC      (Sec. IV-A, V-B)
 *   pastis_substitute_kmers  rows of S: m nearest substitute k-mers   (Sec. IV-B, Alg. 1-3)
 *   pastis_overlap_spgemm    candidates B = A A^T or (A S) A^T        (Sec. IV-A, IV-C)
 *   pastis_align_pairs       Smith-Waterman or x-drop alignment       (Sec. IV-E)
 *   pastis_filter_edges      ANI / coverage filter -> edges           (Sec. IV-F, VI-B)
 *
 * Around it: the row-block form of the product (pastis_overlap_spgemm_rows); the
 * serving form against a resident database (pastis_query_overlap,
 * pastis_align_pairs_qt, pastis_filter_edges_qt); batching (the pass-1 layout and its
 * tuner, pastis_sw_layout_*, pastis_autotune_sw; alignment plans replayed as CUDA
 * graphs, pastis_align_plan_*); a learned prefilter (pastis_pair_features*,
 * pastis_mlp_*, pastis_prefilter_select); the graph variants of Sec. VI-B
 * (PASTIS_SW_SCORE, pastis_ns_edges, pastis_components); a filter that allocates
 * nothing (pastis_filter_edges_static); and the context's profiler and counters.
 *
 * Conventions shared by every call:
 *  - Every pointer named d_* is DEVICE memory owned by the caller; h_* is host
 *    memory.  The library never frees caller memory.  It owns only the workspace
 *    inside a context (grown on demand with cudaMalloc, freed by
 *    pastis_ctx_destroy).
 *  - Work is enqueued on the context's stream.  A call that reports a size to the
 *    host (nnz_out, n_out) synchronises that stream once; the others do not.
 *  - A call that writes a variable-sized result takes `capacity` (records
 *    available at d_out).  If the result does not fit it returns
 *    PASTIS_ERR_CAPACITY, stores the needed count in *n_out and writes nothing to
 *    d_out; calling again with a large enough buffer and the same inputs gives the
 *    result (pastis_overlap_spgemm keeps it and copies it without recomputing).
 *  - No exception crosses the ABI; failures are status codes.  A context is used
 *    by one host thread at a time.
 *  - Residue codes are 0..23 in the order ARNDCQEGHILKMFPSTWYVBZX* (Sec. V-B).
 *    Sequences are concatenated; offsets has n+1 entries, non-decreasing, and a
 *    sequence is at most 65535 residues long (positions are stored as uint16).
 *  - k-mer codes: id = sum_t code(s[p+t]) * 24^(k-1-t), the leftmost residue most
 *    significant (Sec. V-B; RCQ -> 677).  1 <= k <= 6, so ids fit in 32 bits.
 */
#ifndef PASTIS_H
#define PASTIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pastis_status;
enum {
    PASTIS_OK = 0,
    PASTIS_ERR_INVALID_ARG = 1,      /* a null pointer, a size or a parameter out of range */
    PASTIS_ERR_INVALID_RESIDUE = 2,  /* pastis_encode met a byte outside the alphabet      */
    PASTIS_ERR_CAPACITY = 3,         /* d_out too small; *n_out holds the needed count     */
    PASTIS_ERR_OUT_OF_MEMORY = 4,    /* workspace allocation failed                        */
    PASTIS_ERR_CUDA = 5,             /* a CUDA runtime call failed                          */
    PASTIS_ERR_TIMEOUT = 6,          /* a bounded device-side wait ran out                 */
    PASTIS_ERR_UNSUPPORTED = 7,      /* a valid request this library does not implement    */
    PASTIS_ERR_INTERNAL = 8          /* a device-side consistency check failed             */
};

/* Alignment modes (Sec. IV-E; PASTIS_SW_SCORE for the NS weight of Sec. VI-B;
 * PASTIS_SW_FILTERED and PASTIS_XD_FILTERED for the edges of Sec. IV-F only, see
 * pastis_align_pairs). */
enum { PASTIS_SW = 0, PASTIS_XD = 1, PASTIS_SW_SCORE = 2, PASTIS_SW_FILTERED = 3, PASTIS_XD_FILTERED = 4 };

/* Parameters of the method (Sec. VI: k = 6, BLOSUM62, gap open 11, extension 1,
 * x-drop 49, common-k-mer threshold; Sec. IV-F: ANI 30%, coverage 70%).          */
typedef struct pastis_params {
    int32_t k;            /* k-mer length, 1..6                                          */
    int32_t m_subs;       /* substitute k-mers per k-mer, 0 = exact matching, <= 128     */
    int32_t min_shared;   /* candidate iff it shares >= min_shared k-mers; the paper's  */
                          /* "common k-mer threshold t" drops <= t, i.e. min_shared=t+1 */
    int32_t mode;         /* PASTIS_SW, PASTIS_XD or PASTIS_SW_SCORE                     */
    int32_t xdrop;        /* X of the x-drop extension (49)                              */
    int32_t gap_open;     /* a gap of length L costs gap_open + (L-1)*gap_extend         */
    int32_t gap_extend;
    int32_t ani_min_pct;  /* keep iff 100*ident >= ani_min_pct*cols                     */
    int32_t cov_min_pct;  /* and 100*span(shorter) >= cov_min_pct*len(shorter)          */
    int8_t matrix[24 * 24]; /* substitution scores, row-major in alphabet order; must be */
                            /* symmetric, entries in [-64, 63]                            */
} pastis_params;

/* Candidate pair (an entry of B, Sec. IV-A Fig. 3): i < j.  count is the number of
 * shared k-mers (with substitutes: of the orientation kept by symmetrization).  The
 * seeds are the shared k-mers with the two smallest codes, ascending: qpos[s] is the
 * start in sequence i, tpos[s] in sequence j; seed 1 is 0xFFFF when count == 1. 20 B. */
typedef struct pastis_cand {
    int32_t i, j;
    uint32_t count;
    uint16_t qpos[2];
    uint16_t tpos[2];
} pastis_cand;

/* Alignment of candidate (i, j), i the query (rows), j the target.  Spans are
 * half-open: [qb, qe) on i and [tb, te) on j; ident = columns with equal residues,
 * cols = all columns including gap columns.  score == 0 means no positive local
 * alignment and then every other field is 0.  seed_used is the XD seed kept (0 or
 * 1); passes is the filter verdict.  20 B.                                          */
typedef struct pastis_aln {
    int32_t score;
    uint16_t qb, qe, tb, te;
    uint16_t ident, cols;
    uint8_t seed_used, passes;
    uint16_t reserved;
} pastis_aln;

/* Edge of the similarity graph: weight = ANI = ident / cols (IEEE float32 division). */
typedef struct pastis_edge {
    int32_t i, j;
    uint16_t ident, cols;
    int32_t score;
    float weight;
} pastis_edge;

/* The sequence x k-mer matrix A (Sec. IV-A) in two views, all device memory owned by
 * the caller.  Sizes come from pastis_kmat_sizes().
 *   CSR (rows = sequences): row_ptr[n_rows+1]; row_code/row_pos[capacity]: the
 *     distinct k-mers of a row in ascending code order with their smallest start
 *     position (a k-mer repeated in one sequence keeps its first occurrence).
 *   CSC (columns = k-mer codes, dense over all 24^k codes): col_ptr[24^k + 1];
 *     col_seq/col_pos[capacity]: for each code its sequences ascending with the
 *     start position (the posting lists of A^T).
 * pastis_build_kmers fills every array and sets nnz; the other fields are inputs. */
typedef struct pastis_kmat {
    int32_t n_rows;
    int32_t k;
    int64_t capacity;
    int64_t nnz;
    int64_t *row_ptr;
    uint32_t *row_code;
    uint16_t *row_pos;
    uint32_t *col_ptr;
    int32_t *col_seq;
    uint16_t *col_pos;
} pastis_kmat;

typedef struct pastis_ctx pastis_ctx;

/* ---- context ------------------------------------------------------------------ */

/* Creates a context on `device` that enqueues on `stream` (a cudaStream_t; NULL is
 * the legacy default stream).  The stream must outlive the context.              */
pastis_status pastis_ctx_create(pastis_ctx **ctx, int device, void *stream);
pastis_status pastis_ctx_destroy(pastis_ctx *ctx);
const char *pastis_status_string(pastis_status s);
/* Kept results.  A product with substitutes keeps the AS matrix it built (Sec. IV-C)
 * together with a copy of A's rows; a later product whose A has the same rows (compared
 * on the device, one read of both copies) and the same k, m and matrix reuses it, so the
 * row blocks of one job build S and AS once.  The last product's candidates are kept for
 * the two-phase size protocol.  pastis_ctx_forget drops both, so the next call computes
 * everything again (the workspace stays allocated).                                 */
pastis_status pastis_ctx_forget(pastis_ctx *ctx);
/* Bytes of workspace the context holds now. */
int64_t pastis_ctx_workspace_bytes(const pastis_ctx *ctx);
/* Kernel launches the context has issued since creation (for accounting). */
int64_t pastis_ctx_launch_count(const pastis_ctx *ctx);
/* Per-kernel timing: with enable != 0 the context brackets its main kernels with CUDA
 * events on its stream (this adds event records, not synchronisation).
 * pastis_ctx_profile_read synchronises the stream and writes one line per kernel name,
 * "name launches total_ms", into buf (at most len bytes, NUL-terminated); it returns
 * the bytes written.  Enabling again clears the totals.                             */
pastis_status pastis_ctx_profile(pastis_ctx *ctx, int enable);
int32_t pastis_ctx_profile_read(pastis_ctx *ctx, char *buf, int32_t len);
/* Work counters accumulated while profiling is on (cleared when it is enabled), for the
 * roofline of the overlap product: h_out[0] = posting entries visited (products),
 * [1] = left-operand entries of the rows formed (each once per row), [2] = candidate
 * records written, [3] = radix-sort element passes of the k-mer matrix builds (A and AS:
 * elements sorted x 8-bit digit passes).  Entries past the fourth are 0.  Synchronises
 * the stream.                                                                             */
#define PASTIS_STATS 4
pastis_status pastis_ctx_stats(pastis_ctx *ctx, int64_t *h_out, int32_t n);

/* ---- integer-pipe throughput probe (a measurement of the GPU, not of the method) ----
 * Runs one instruction kind (or the instruction mix of the Smith-Waterman pass-1
 * recurrence, PASTIS_PROBE_SW_MIX) in many independent dependency chains on every SM,
 * blocks_per_sm CTAs of 256 threads per SM, all resident at once, for `iters`
 * iterations, and stores the measured rate in warp-instructions per SM clock (clock64
 * inside each CTA; the slowest CTA counts) in *h_warp_inst_per_clk_sm.  The alignment
 * roofline divides by this measured rate.  UNSUPPORTED when blocks_per_sm CTAs do not
 * fit on an SM.  Synchronises.                                                       */
enum {
    PASTIS_PROBE_VIADDMAX_S16X2 = 0,   /* max(a + b, c) per 16-bit half        */
    PASTIS_PROBE_VIMAX3_S16X2_RELU = 1,/* max(a, b, c, 0) per 16-bit half      */
    PASTIS_PROBE_VADD2 = 2,            /* a + b per 16-bit half                */
    PASTIS_PROBE_PRMT = 3,             /* byte permute                         */
    PASTIS_PROBE_IMAD = 4,             /* 32-bit multiply-add                  */
    PASTIS_PROBE_IMAX = 5,             /* 32-bit signed maximum                */
    PASTIS_PROBE_LOP3 = 6,             /* (a & b) | c; the compiler folds steps */
    PASTIS_PROBE_IADD = 7,             /* 32-bit add                           */
    PASTIS_PROBE_SW_MIX = 8,           /* the pass-1 recurrence mix            */
    PASTIS_PROBE_MAX3_ADD2 = 9         /* 16x2 three-way max and 16x2 add, 1:1 */
};
pastis_status pastis_probe_int_throughput(pastis_ctx *ctx, int32_t kind, int32_t blocks_per_sm, int32_t iters,
                                          double *h_warp_inst_per_clk_sm);

/* ---- a1: encode (Sec. V-B) ---------------------------------------------------- */

/* d_ascii[n_bytes] letters -> d_codes[n_bytes] codes 0..23.  Any byte outside the
 * 24 upper-case letters of the alphabet gives PASTIS_ERR_INVALID_RESIDUE, and
 * *bad_index (if not NULL) receives the first offending index.  Synchronises.     */
pastis_status pastis_encode(pastis_ctx *ctx, const uint8_t *d_ascii, int64_t n_bytes,
                            uint8_t *d_codes, int64_t *bad_index);

/* ---- a2-a3: k-mers and A (Sec. IV-A, Sec. V-B) --------------------------------- */

/* Sizes to allocate for A over n sequences with R residues in total: capacity bounds
 * the (row, k-mer) entries that can occur (R: each residue starts at most one window)
 * and col_ptr_len = 24^k + 1.                                                      */
pastis_status pastis_kmat_sizes(int32_t n, int64_t total_residues, int32_t k,
                                int64_t *capacity, int64_t *col_ptr_len);

/* Builds A from d_codes/d_offsets (n sequences) with a device radix sort: CSR
 * rows, then CSC posting lists.  A->n_rows, A->k, A->capacity and the array
 * pointers are inputs; A->nnz and *nnz_out receive the entry count.  A capacity
 * below the number of windows gives PASTIS_ERR_CAPACITY.  Synchronises.            */
pastis_status pastis_build_kmers(pastis_ctx *ctx, const uint8_t *d_codes,
                                 const int64_t *d_offsets, int32_t n, int32_t k,
                                 pastis_kmat *A, int64_t *nnz_out);

/* ---- a4: substitute k-mers (Sec. IV-B, Alg. 1-3) -------------------------------- */

/* For each of n_roots k-mer codes r, row r of S: d_sub_code[r*(m+1) + 0] = r with
 * distance 0, then the m k-mers q != r nearest to r, ascending by (distance, code).
 * distance(r, q) = sum_t (M[r_t][r_t] - M[r_t][q_t]) (the expense matrix E of
 * Sec. IV-B; not symmetric).  Ties at equal distance take the smaller code.        */
pastis_status pastis_substitute_kmers(pastis_ctx *ctx, const uint32_t *d_roots,
                                      int64_t n_roots, const pastis_params *params,
                                      uint32_t *d_sub_code, int32_t *d_sub_dist);

/* ---- a5-a7: candidate discovery (Sec. IV-A, IV-C) ------------------------------ */

/* Candidates i < j of the overlap product.  params->m_subs == 0: B = A A^T with the
 * semiring that counts shared k-mers and keeps two seeds (Sec. IV-A).  m_subs > 0:
 * S is formed for the k-mers present, AS(i, s) keeps the start of the k-mer of i
 * nearest to s (smaller start on ties), both orientations (AS)_i.A_j and (AS)_j.A_i
 * are formed, and the pair keeps the orientation sharing more (i->j on ties) --
 * symmetrization (Sec. VI-A).  Pairs with count < min_shared are dropped.  Output
 * sorted by (i, j).  Synchronises.                                                   */
pastis_status pastis_overlap_spgemm(pastis_ctx *ctx, const pastis_kmat *A,
                                    const pastis_params *params, pastis_cand *d_out,
                                    int64_t capacity, int64_t *n_out);

/* The rows row_begin <= i < row_end of the same product (every j > i): a block of
 * queries against the whole set, for batched or partial formation of B (the paper's
 * Sec. VII names partial formation of the output as the way to cap memory).  The
 * result equals the matching slice of pastis_overlap_spgemm's.  Synchronises.        */
pastis_status pastis_overlap_spgemm_rows(pastis_ctx *ctx, const pastis_kmat *A,
                                         const pastis_params *params, int32_t row_begin,
                                         int32_t row_end, pastis_cand *d_out, int64_t capacity,
                                         int64_t *n_out);

/* Serving form: query sequences (rows of Q) against a database (columns = every
 * sequence of DB, not only j > i); pair (i, j) names query i and database entry j.
 * Exact k-mers only (params->m_subs == 0, else PASTIS_ERR_UNSUPPORTED).  Q and DB are
 * each built by pastis_build_kmers.  Output sorted by (i, j).  Synchronises.        */
pastis_status pastis_query_overlap(pastis_ctx *ctx, const pastis_kmat *Q, const pastis_kmat *DB,
                                   const pastis_params *params, pastis_cand *d_out, int64_t capacity,
                                   int64_t *n_out);

/* ---- a8-a9: alignment (Sec. IV-E) ---------------------------------------------- */

/* One record per candidate, d_out[n_pairs].
 * PASTIS_SW: Smith-Waterman, affine gaps, seeds ignored.  The end is the first
 *   maximum in row-major order (rows = residues of i); the alignment is the one a
 *   traceback from it selects when it prefers diagonal > vertical gap > horizontal
 *   gap in H, and gap open over gap extension.
 * PASTIS_XD: from each seed, seed score plus gapped x-drop extensions to the right
 *   and to the left (antidiagonal order; a cell dies when H < best - xdrop); among
 *   the seeds whose alignment passes the filter the higher score (first seed on
 *   ties) is kept, otherwise the best score with passes = 0.
 * PASTIS_SW_SCORE: the Smith-Waterman score and end only (what the NS weight needs;
 *   no traceback): score, qe, te as in PASTIS_SW; qb, tb, ident, cols, passes are 0.
 * PASTIS_SW_FILTERED: what the filter needs (Sec. IV-F).  A pair that passes gets the
 *   record of PASTIS_SW; a pair that fails gets PASTIS_SW's score, qe and te with qb,
 *   tb, ident, cols and passes 0.  pastis_filter_edges gives the same edges as after
 *   PASTIS_SW.  Pairs whose end (or the rectangle that bounds their path) leaves less
 *   than the coverage bound on the shorter sequence are never traced back.
 * PASTIS_XD_FILTERED: the same for x-drop.  A pair that passes gets the record of
 *   PASTIS_XD; a pair that fails gets PASTIS_XD's score, qe, te and seed_used with qb,
 *   tb, ident, cols and passes 0.  Every extension is first computed without carried
 *   statistics; only the seeds whose spans pass the coverage test are extended again
 *   with them.
 * d_offsets has n_seqs+1 entries; a pair naming a sequence outside [0, n_seqs), or
 * (XD) a seed that does not fit its sequence, gives PASTIS_ERR_INVALID_ARG before any
 * alignment runs.  d_cells (optional, device int64) accumulates the DP cells computed
 * (|q|*|t| per SW pair; computed antidiagonal cells for XD).  Synchronises.         */
pastis_status pastis_align_pairs(pastis_ctx *ctx, const uint8_t *d_codes,
                                 const int64_t *d_offsets, int32_t n_seqs,
                                 const pastis_cand *d_pairs, int64_t n_pairs,
                                 const pastis_params *params, pastis_aln *d_out,
                                 int64_t *d_cells);

/* The same with the queries' and targets' residues in separate arrays: pair (i, j)
 * aligns query i of (d_qcodes, d_qoffsets[n_q+1]) with target j of (d_tcodes,
 * d_toffsets[n_t+1]) -- the serving form, database resident and queries per batch.  */
pastis_status pastis_align_pairs_qt(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets,
                                    int32_t n_q, const uint8_t *d_tcodes, const int64_t *d_toffsets,
                                    int32_t n_t, const pastis_cand *d_pairs, int64_t n_pairs,
                                    const pastis_params *params, pastis_aln *d_out, int64_t *d_cells);

/* ---- batching: the Smith-Waterman tile layout and its tuner -----------------------
 * Pass 1 of PASTIS_SW / PASTIS_SW_SCORE computes a query of m residues in stripes of
 * 32 lanes x LR rows (LR 2..16), two pairs per warp in the 16-bit halves of every
 * register.  By default it takes as few stripes as 16 rows per lane allow; a layout
 * sets, per query-length bin (bin = (m-1) / 32, the last bin taking every longer
 * query), either 0..PASTIS_SW_MAX_EXTRA extra stripes, which pad fewer rows but sweep
 * the target more often, or PASTIS_SW_INT32: the bin's pairs take one pair per warp in
 * 32-bit lanes (the whole-matrix path that also serves pairs whose scores could
 * overflow 16 bits).  The layout is a speed choice only: every output of every entry
 * point is the same under every layout.                                             */
#define PASTIS_SW_BINS 64
#define PASTIS_SW_BIN_WIDTH 32
#define PASTIS_SW_MAX_EXTRA 2
#define PASTIS_SW_INT32 3

/* Sets the context's layout from h_extra[PASTIS_SW_BINS] (host; NULL = the default,
 * all 0).  A value other than 0..PASTIS_SW_MAX_EXTRA or PASTIS_SW_INT32 gives
 * PASTIS_ERR_INVALID_ARG and leaves the layout unchanged.  pastis_sw_layout_get copies
 * the current one to h_extra.                                                        */
pastis_status pastis_sw_layout_set(pastis_ctx *ctx, const uint8_t *h_extra);
pastis_status pastis_sw_layout_get(const pastis_ctx *ctx, uint8_t *h_extra);

/* The autotuner: runs the score-and-end alignment of the given pairs (the arguments
 * of pastis_align_pairs_qt; a sample of the workload's candidates) once per uniform
 * layout 0..PASTIS_SW_MAX_EXTRA and PASTIS_SW_INT32, `reps` times each, with the SM
 * cycles of every query's pass-1 work and of every pair's 32-bit work summed per
 * length bin; each bin takes the layout with the fewest cycles when it beats the
 * default by at least 2%, else the default.  The chosen layout is set on the context
 * and copied to h_extra (optional, PASTIS_SW_BINS bytes); h_cycles (optional, host,
 * PASTIS_SW_BINS * (PASTIS_SW_MAX_EXTRA + 2) int64, [x * BINS + bin], x = 0..2 the
 * extra stripes, x = 3 the 32-bit lanes) receives the measured cycles.  params->mode must be PASTIS_SW or PASTIS_SW_SCORE
 * (PASTIS_ERR_UNSUPPORTED otherwise).  Validation and errors as
 * pastis_align_pairs_qt; the layout is unchanged on error.  Synchronises.           */
pastis_status pastis_autotune_sw(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets,
                                 int32_t n_q, const uint8_t *d_tcodes, const int64_t *d_toffsets,
                                 int32_t n_t, const pastis_cand *d_pairs, int64_t n_pairs,
                                 const pastis_params *params, int32_t reps, uint8_t *h_extra,
                                 int64_t *h_cycles);

/* ---- batching: the x-drop lane layout -------------------------------------------------
 * The extensions of Sec. IV-E's x-drop (PASTIS_XD: each with its carried statistics;
 * PASTIS_XD_FILTERED: first every extension's score, end and cells, then the carried
 * statistics of the seeds that may pass) run in 16-bit lanes with `per_warp`
 * extensions side by side in each warp (1, 2 or 4: one window of 128 diagonals over 32,
 * 16 or 8 lanes), or in 32-bit lanes, one extension per warp (per_warp = 0).
 * Extensions the 16-bit form cannot hold run in 32-bit lanes whatever the setting: gap
 * open or extend above 128, X above 30,000, the largest substitution score times the
 * shorter side of the extension above 30,000, a side of length 0, or a computed
 * antidiagonal wider than 64 cells.  A speed choice only: every output is the same
 * under every setting.  A context starts with PASTIS_XD_DEFAULT_PER_WARP.
 * pastis_xd_layout_set gives PASTIS_ERR_INVALID_ARG for any other value and leaves the
 * setting unchanged; pastis_xd_layout_get returns it (-1 for a NULL context).        */
#define PASTIS_XD_DEFAULT_PER_WARP 4
pastis_status pastis_xd_layout_set(pastis_ctx *ctx, int32_t per_warp);
int32_t pastis_xd_layout_get(const pastis_ctx *ctx);

/* The x-drop layout tuner: runs the x-drop of params->mode on the given pairs (the
 * arguments of pastis_align_pairs_qt; a sample of the workload's candidates) under each setting,
 * 0, 1, 2 and 4, `reps` times each, every call timed by CUDA events on the context's
 * stream.  The fastest setting is set on the context when it beats the current one by
 * 2% or more (else the current one stays) and copied to *h_per_warp (optional); h_ms
 * (optional, host, 4 doubles) receives each setting's best time in milliseconds, in
 * the order 0, 1, 2, 4.  params->mode must be PASTIS_XD or PASTIS_XD_FILTERED
 * (PASTIS_ERR_UNSUPPORTED otherwise).  Validation and errors as
 * pastis_align_pairs_qt; the setting is unchanged on error.  Synchronises.          */
pastis_status pastis_autotune_xd(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets,
                                 int32_t n_q, const uint8_t *d_tcodes, const int64_t *d_toffsets,
                                 int32_t n_t, const pastis_cand *d_pairs, int64_t n_pairs,
                                 const pastis_params *params, int32_t reps, int32_t *h_per_warp,
                                 double *h_ms);

/* ---- batching: alignment plans replayed as CUDA graphs ------------------------------
 * A plan captures the whole alignment of one batch (the input checks, then pass 1-3 of
 * PASTIS_SW / PASTIS_SW_SCORE or the x-drop extensions and their combination) once, as
 * a CUDA graph over buffers of fixed capacity, against a target set that stays resident
 * (the serving form: the database).  Each run copies the batch into the plan's buffers,
 * writes its counts to device memory and launches the graph: one launch and one
 * synchronisation instead of a launch per kernel and a synchronisation per stage.  The
 * kernels are the ones pastis_align_pairs_qt runs, sized for the capacity (persistent
 * grids, scans over the capacity with zero counts past the batch), so every record
 * equals pastis_align_pairs_qt's on the same batch.
 *
 * pastis_align_plan_create: ctx supplies the device, the stream (the plan runs on it)
 *   and the pass-1 and x-drop layouts at this moment; the plan owns a private workspace.  Targets
 *   d_tcodes / d_toffsets[n_t+1] (device; they must stay valid and unchanged while the
 *   plan lives) are checked once: a code >= 24 gives PASTIS_ERR_INVALID_RESIDUE, a
 *   target longer than max_len PASTIS_ERR_INVALID_ARG.  Capacities: max_q queries,
 *   max_qres query residues, max_pairs pairs, max_len residues per query or target
 *   (<= 65535).  params is copied (every mode).  Synchronises.
 * pastis_align_plan_run: queries d_qcodes (device) with offsets h_qoffsets[n_q+1] on the
 *   HOST (h_qoffsets[0] = 0, non-decreasing, else PASTIS_ERR_INVALID_ARG), pairs
 *   d_pairs[n_pairs] (device) as for pastis_align_pairs_qt, records to d_out[n_pairs]
 *   (device).  A batch above a capacity (n_q, n_pairs, residues, a query longer than
 *   max_len) gives PASTIS_ERR_CAPACITY before any work; a pair naming a sequence
 *   outside the batch or the targets (or an x-drop seed that does not fit) gives
 *   PASTIS_ERR_INVALID_ARG, a query code >= 24 PASTIS_ERR_INVALID_RESIDUE; then the
 *   alignment kernels have done nothing, d_out is untouched and the plan stays usable.
 *   Synchronises.
 * pastis_align_plan_destroy: waits for the plan's stream and frees everything.
 * pastis_align_plan_graph_nodes: nodes of the captured graph (-1 on error).         */
typedef struct pastis_align_plan pastis_align_plan;
pastis_status pastis_align_plan_create(pastis_ctx *ctx, const uint8_t *d_tcodes, const int64_t *d_toffsets,
                                       int32_t n_t, int32_t max_q, int64_t max_qres, int64_t max_pairs,
                                       int32_t max_len, const pastis_params *params, pastis_align_plan **out);
pastis_status pastis_align_plan_run(pastis_align_plan *plan, const uint8_t *d_qcodes, const int64_t *h_qoffsets,
                                    int32_t n_q, const pastis_cand *d_pairs, int64_t n_pairs, pastis_aln *d_out);
pastis_status pastis_align_plan_destroy(pastis_align_plan *plan);
int64_t pastis_align_plan_graph_nodes(const pastis_align_plan *plan);

/* ---- a10: similarity filter (Sec. IV-F, VI-B) ----------------------------------- */

/* Keeps pair p iff cols > 0, 100*ident >= ani*cols and 100*span >= cov*len, span and
 * len taken on the shorter sequence (i on equal lengths).  Edges keep pair order.
 * Synchronises.                                                                     */
pastis_status pastis_filter_edges(pastis_ctx *ctx, const int64_t *d_offsets, int32_t n_seqs,
                                  const pastis_cand *d_pairs, const pastis_aln *d_alns,
                                  int64_t n_pairs, const pastis_params *params,
                                  pastis_edge *d_out, int64_t capacity, int64_t *n_out);

/* ---- learned prefilter (an extension; no counterpart in the paper's method) ----
 * A 16 -> 256 -> 256 -> 1 MLP over per-pair features predicts whether a candidate's
 * alignment will pass the filter, so that predicted failures skip alignment.  It is
 * the learned analogue of the paper's common-k-mer threshold (Sec. VI, which trades
 * 2-3% recall for > 90% fewer alignments, Sec. VI-B).  Weights are float32 masters
 * with bf16 copies used by the tensor-core kernels (f32 accumulation).  All buffers
 * are caller-owned device memory; sizes: NW1 = 16*256, NW2 = 256*256, NW3 = 256.
 * Layouts: w1[i*256 + o], w2[i*256 + o] (input-major), w3[i], b1[256], b2[256], b3[1];
 * grad / adam_m / adam_v each hold NW1 + 256 + NW2 + 256 + NW3 + 1 floats laid out as
 * w1, b1, w2, b2, w3, b3.                                                               */
typedef struct pastis_mlp {
    float *w1, *b1, *w2, *b2, *w3, *b3;
    void *w1b, *w2b, *w3b;       /* __nv_bfloat16 copies of w1, w2, w3 */
    float *grad, *adam_m, *adam_v;
    int64_t step;                /* Adam steps taken (updated by train_step) */
} pastis_mlp;

/* Features of each candidate, d_x[n_pairs * 16] as bf16 (row-major). */
pastis_status pastis_pair_features(pastis_ctx *ctx, const uint8_t *d_codes, const int64_t *d_offsets,
                                   const pastis_cand *d_pairs, int64_t n_pairs,
                                   const pastis_params *params, void *d_x);

/* The same with the queries' and targets' residues in separate arrays (serving form:
 * pair (i, j) is query i against target j). */
pastis_status pastis_pair_features_qt(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets,
                                      const uint8_t *d_tcodes, const int64_t *d_toffsets, const pastis_cand *d_pairs,
                                      int64_t n_pairs, const pastis_params *params, void *d_x);
/* Logits d_logits[n] of d_x[n * 16] (bf16).  Does not synchronise. */
pastis_status pastis_mlp_forward(pastis_ctx *ctx, const pastis_mlp *net, const void *d_x, int64_t n,
                                 float *d_logits);
/* One Adam step (lr, beta 0.9/0.999) on the weighted logistic loss of d_x[n * 16]
 * against labels d_y[n] in {0, 1}; positives weigh pos_weight.  n <= 2^22.  *d_loss
 * (device, optional) receives the mean loss.  Does not synchronise.                */
pastis_status pastis_mlp_train_step(pastis_ctx *ctx, pastis_mlp *net, const void *d_x, const float *d_y,
                                    int64_t n, float lr, float pos_weight, float *d_loss);
/* The candidates whose logit >= threshold, in input order (capacity protocol as for
 * the other variable-size outputs).  Synchronises.                                   */
pastis_status pastis_prefilter_select(pastis_ctx *ctx, const pastis_cand *d_pairs, const float *d_logits,
                                      int64_t n_pairs, float threshold, pastis_cand *d_out,
                                      int64_t capacity, int64_t *n_out);

/* The filter with queries and targets in separate offset arrays (serving form). */
pastis_status pastis_filter_edges_qt(pastis_ctx *ctx, const int64_t *d_qoffsets, int32_t n_q,
                                     const int64_t *d_toffsets, int32_t n_t, const pastis_cand *d_pairs,
                                     const pastis_aln *d_alns, int64_t n_pairs, const pastis_params *params,
                                     pastis_edge *d_out, int64_t capacity, int64_t *n_out);

/* ---- variants of the graph (Sec. VI-B) ------------------------------------------ */

/* NS edges: every pair with a positive score becomes an edge (i, j, ident, cols, score,
 * weight = score / min(|s_i|, |s_j|) as a correctly rounded float32), in pair order.
 * The NS weight needs no traceback, so alignments from PASTIS_SW_SCORE suffice; the
 * ANI and coverage tests need one and are not applied.  Capacity protocol and errors
 * as pastis_filter_edges.  Synchronises.                                              */
pastis_status pastis_ns_edges(pastis_ctx *ctx, const int64_t *d_offsets, int32_t n_seqs,
                              const pastis_cand *d_pairs, const pastis_aln *d_alns, int64_t n_pairs,
                              pastis_edge *d_out, int64_t capacity, int64_t *n_out);

/* Connected components of the graph on n_seqs vertices whose edges are d_edges[n_edges]
 * (only i and j are read), for the components-as-families variant (Sec. VI-B).
 * d_labels[n_seqs] receives, for each vertex, the smallest vertex of its component, so
 * the result does not depend on the order of the edges.  An endpoint outside
 * [0, n_seqs) gives PASTIS_ERR_INVALID_ARG; PASTIS_ERR_INTERNAL if a bounded union-find
 * walk runs out (it cannot on a valid input).  Synchronises.                           */
pastis_status pastis_components(pastis_ctx *ctx, int32_t n_seqs, const pastis_edge *d_edges, int64_t n_edges,
                                int32_t *d_labels);

/* ---- the filter without allocation ------------------------------------------------
 * The paper has no counterpart of this call.  It gives exactly what pastis_filter_edges
 * gives (the same keep rule, the same edges, the same pair order, bit for bit) for
 * callers that may not allocate device memory: a worker whose device memory is all
 * committed (a serving slot admitted against a fixed memory budget), or one that must
 * not call cudaFree, which waits for the whole device and so stalls other streams.
 * It takes no context (creating one allocates its workspace) and neither calls
 * cudaMalloc/cudaFree nor any library that allocates: its scratch is one fixed device
 * array of PASTIS_FILTER_STATIC_SCRATCH_BYTES inside this library (a kept count and an
 * offset per tile of 1,024 pairs, an error word, the total), which every GPU that loads
 * the library holds until the process exits.
 *
 * stream      a cudaStream_t (NULL: the legacy default stream) of the current device;
 *             every d_* pointer is device memory of that device, owned by the caller.
 * d_offsets   n_seqs + 1 offsets of the sequences that pair indices i, j refer to.
 * d_pairs, d_alns   n_pairs candidates and their alignments (pastis_align_pairs order).
 * d_out, capacity   room for edges; *n_out receives the number of edges.
 * Limits and errors: n_pairs > PASTIS_FILTER_STATIC_MAX_PAIRS returns
 * PASTIS_ERR_UNSUPPORTED before any work; a pair index outside [0, n_seqs) returns
 * PASTIS_ERR_INVALID_ARG; too small a capacity returns PASTIS_ERR_CAPACITY with the
 * needed count in *n_out and nothing written.  Nothing the caller passes has to start
 * at zero; the call clears its own error word first.
 * Set-up: the first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it; make that first call
 * before any stream capture begins.  A lookup that fails returns PASTIS_ERR_CUDA and is
 * not kept: the next call on that device tries again.  Every call after a successful
 * lookup does no set-up.
 * Concurrency: all calls on one device share the one scratch array, so calls that
 * overlap in time (from several threads, or on several streams) race and corrupt each
 * other's result; the caller runs them one at a time per device.
 * Synchronises the stream twice (to read the total, and at the end).                   */
#define PASTIS_FILTER_STATIC_MAX_PAIRS 4194304
#define PASTIS_FILTER_STATIC_SCRATCH_BYTES 33024
pastis_status pastis_filter_edges_static(void *stream, const int64_t *d_offsets, int32_t n_seqs,
                                         const pastis_cand *d_pairs, const pastis_aln *d_alns,
                                         int64_t n_pairs, const pastis_params *params,
                                         pastis_edge *d_out, int64_t capacity, int64_t *n_out);

#ifdef __cplusplus
}
#endif
#endif /* PASTIS_H */
