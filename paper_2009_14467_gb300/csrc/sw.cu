// a8: Smith-Waterman of candidate pairs (Sec. IV-E, Sec. VI), three passes.
//
// Recurrences (a gap of length L costs open + (L-1)*extend):
//   E(i,j) = max(H(i,j-1) - o, E(i,j-1) - e)     F(i,j) = max(H(i-1,j) - o, F(i-1,j) - e)
//   H(i,j) = max(0, H(i-1,j-1) + s(q_i, t_j), F(i,j), E(i,j))
// Reported: the score S, the end = the first maximum in row-major order, and the
// alignment a traceback from the end selects when it prefers the diagonal, then F,
// then E, and a gap open over an extension (its begin, identities, columns).
//
// Pass 1 (the whole matrix, every pair): score and end only.  A warp owns a pair;
//   lane l owns 16 consecutive query rows and at step s computes column j = s - l,
//   taking the H/F of the row above from lane l-1 (__shfl_up_sync).  Scores come from
//   a query profile in shared memory (int16, [target residue][query row]) shared by
//   every warp of the CTA: the CTA works through a run of pairs with the same query
//   (candidate lists are grouped by i).  The end is tracked with one key per cell,
//   key = H * 2^16 + (65535 - i): the largest key is the largest H on the smallest
//   row, and a lane keeps the first column where its largest key appears, which is
//   the row-major first maximum.  Queries longer than 512 rows go in stripes whose
//   last row is handed on through a per-warp buffer.
// Pass 2 (right after pass 1, same warp; a region around the path): an anchored DP
//   over the reversed prefixes from the end (ei, ej).  A suffix of the traced path
//   starting on row i scores S minus the forward value before it, which is at most
//   the largest H pass 1 met on row i-1's 16-row block; cells below that threshold
//   die, the path's suffixes all survive, and the cells reaching S bound the begin.
//   Their extent gives a rectangle that contains the whole traced path.
// Pass 3 (that rectangle): the DP again with zero boundaries; each state carries its
//   begin cell and (identities << 16 | matched columns) along the predecessor a
//   traceback would take.  Inside a rectangle holding the path, the path's cells keep
//   their values and every choice along it is the same, so the carry at the end cell
//   is the traceback's.  cols = span_q + span_t - matched.
// Scores that could reach 2^15 (11 * min length >= 32768 with BLOSUM62) take pass 3
// over the whole matrix with the end tracked there instead (all int32 either way).
#include <algorithm>

#include "internal.cuh"

namespace {

constexpr int NEG = -1000000000;
constexpr int SW_THREADS = 256;
constexpr int SW_WARPS = SW_THREADS / 32;
constexpr int LR = 16;                     // query rows per lane in pass 1
constexpr int STRIPE1 = 32 * LR;           // rows per stripe in pass 1
constexpr int PAD_SCORE = -30000;
constexpr int SEG_MAX = 64;                // pairs per scheduling segment

struct sw_score_out {                      // pass 1 result per pair
    int32_t score;
    int32_t end_i, end_j;
    int32_t rect_i, rect_j;                // pass 2: start of the bounding rectangle
    int32_t big;                           // scores may not fit the pass-1 key
};

// ---------------------------------------------------------------------------------
// segments: runs of pairs with the same query, at most SEG_MAX long
// ---------------------------------------------------------------------------------
__global__ void k_seg_flags(const pastis_cand *pairs, int64_t n, uint32_t *flags) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    flags[p] = (p == 0 || (p % SEG_MAX) == 0 || pairs[p].i != pairs[p - 1].i) ? 1u : 0u;
}

__global__ void k_seg_starts(const uint32_t *flags, const uint32_t *off, int64_t n, int64_t *seg_start) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n && flags[p]) seg_start[off[p]] = p;
    if (p == n - 1) seg_start[off[p] + flags[p]] = n;
}

// ---------------------------------------------------------------------------------
// pass 1
// ---------------------------------------------------------------------------------
struct stripe1_cell { int32_t h, f; };

__device__ __forceinline__ int sx_lo(uint32_t w) { return (int)(int16_t)(w & 0xFFFF); }
__device__ __forceinline__ int sx_hi(uint32_t w) { return (int)w >> 16; }

// LR query rows per lane (even, 2..16, from the query length, so that the padding past
// the query stays small); a stripe is 32 * LR rows.  bm4[g] receives, for every pair of
// rows, the largest H of the lane block that holds it (an upper bound per row).
template <int LR>
__device__ void score_warp(const int16_t *__restrict__ prof, int prow, const uint8_t *__restrict__ t, int m,
                           int n, int o, int e, stripe1_cell *scratch, int sstride, int16_t *bm4, int *best_h,
                           int *best_i, int *best_j) {
    constexpr int STRIPE = 32 * LR;
    const int lane = threadIdx.x & 31;
    int bestkey = 65535, bestj = 0;
    const int nstripes = (m + STRIPE - 1) / STRIPE;
    for (int stripe = 0; stripe < nstripes; ++stripe) {
        const int row0 = stripe * STRIPE + lane * LR;
        // key addend: 65535 - i on real rows; rows past the query get INT_MIN, so
        // their keys (H * 2^16 + INT_MIN < 0) never win
        int H[LR], E[LR], ck[LR];
#pragma unroll
        for (int r = 0; r < LR; ++r) {
            const int i = row0 + r;
            H[r] = 0;
            E[r] = NEG;
            ck[r] = i < m ? 65535 - i : (int)0x80000000;
        }
        int dtop = 0;                                  // H(row0-1, j-1)
        int out_h = 0, out_f = NEG, out_t = 0;
        const stripe1_cell *in_buf = scratch + (size_t)(stripe & 1) * sstride;
        stripe1_cell *out_buf = scratch + (size_t)((stripe + 1) & 1) * sstride;
        const bool last = stripe + 1 == nstripes;
        const int16_t *prow0 = prof + row0;
        int blockkey = 0;                              // largest key of this lane's rows
        for (int s = 0; s < n + 31; ++s) {
            const int j = s - lane;
            int up_h = __shfl_up_sync(0xffffffffu, out_h, 1);
            int up_f = __shfl_up_sync(0xffffffffu, out_f, 1);
            int tj = __shfl_up_sync(0xffffffffu, out_t, 1);
            if (lane == 0 && j < n) {
                tj = t[j];
                if (stripe == 0) { up_h = 0; up_f = NEG; }
                else { const stripe1_cell c = in_buf[j]; up_h = c.h; up_f = c.f; }
            }
            if (j >= 0 && j < n) {
                uint32_t ws[LR / 2];
                if (LR % 8 == 0) {
                    const uint4 *pv = reinterpret_cast<const uint4 *>(prow0 + tj * prow);
#pragma unroll
                    for (int k = 0; k < LR / 8; ++k) {
                        const uint4 v = pv[k];
                        ws[4 * k] = v.x; ws[4 * k + 1] = v.y; ws[4 * k + 2] = v.z; ws[4 * k + 3] = v.w;
                    }
                } else if (LR % 4 == 0) {
                    const uint2 *pv = reinterpret_cast<const uint2 *>(prow0 + tj * prow);
#pragma unroll
                    for (int k = 0; k < LR / 4; ++k) {
                        const uint2 v = pv[k];
                        ws[2 * k] = v.x; ws[2 * k + 1] = v.y;
                    }
                } else {
                    const uint32_t *pv = reinterpret_cast<const uint32_t *>(prow0 + tj * prow);
#pragma unroll
                    for (int k = 0; k < LR / 2; ++k) ws[k] = pv[k];
                }
                int sk = 0;
                int hprev = dtop;                      // H(i-1, j-1) for the row being done
                int ha = up_h, f = up_f;               // H(i-1, j), F(i-1, j)
#pragma unroll
                for (int r = 0; r < LR; ++r) {
                    const int sc = (r & 1) ? sx_hi(ws[r >> 1]) : sx_lo(ws[r >> 1]);
                    const int d = hprev + sc;
                    const int ev = max(H[r] - o, E[r] - e);
                    f = max(ha - o, f - e);
                    const int h = max(__vimax3_s32(d, ev, f), 0);
                    hprev = H[r];
                    H[r] = h;
                    E[r] = ev;
                    ha = h;
                    sk = max(sk, h * 65536 + ck[r]);
                }
                if (sk > bestkey) { bestkey = sk; bestj = j; }
                blockkey = max(blockkey, sk);
                dtop = up_h;
                out_h = ha; out_f = f; out_t = tj;
                if (lane == 31 && !last) out_buf[j] = stripe1_cell{ha, f};
            }
        }
#pragma unroll
        for (int g = 0; g < LR / 2; ++g) bm4[(row0 >> 1) + g] = (int16_t)(blockkey >> 16);
        __syncwarp();
    }
    // row-major first maximum across the warp: the largest key (ties cannot cross lanes)
    bestkey = max(bestkey, 65535);
    const int top = __reduce_max_sync(0xffffffffu, bestkey);
    const unsigned who = __ballot_sync(0xffffffffu, bestkey == top);
    *best_h = top >> 16;
    *best_i = 65535 - (top & 0xFFFF);
    *best_j = __shfl_sync(0xffffffffu, bestj, __ffs(who) - 1);
}

// ---------------------------------------------------------------------------------
// pass 2: bounding rectangle of the traced path, by an anchored DP over the reversed
// prefixes in which cells below 0 die
// ---------------------------------------------------------------------------------
constexpr int WIN = 64;           // cells of one antidiagonal kept in shared memory

// The suffix of the traced path that starts on forward row i scores S minus the
// forward value of the path state before it, which sits on row i-1; that value is at
// most bm4[(i-1)/2], the largest H pass 1 saw on those rows.  When the split falls
// inside a gap run, the reverse DP charges the suffix's part of the run an open
// instead of an extension, so its reverse value can be lower by o - e.  A reverse cell
// whose first row is i therefore dies below S - bm4[(i-1)/2] - (o - e) (bm = 0 above
// row 0); every suffix of the path meets the bound, so the path survives, and the
// cells reaching S bound its begin.  Three antidiagonals of H, E, F live in a circular
// window of WIN cells per array; a live band wider than that returns false and the
// caller falls back to the whole up-left rectangle.
__device__ bool bound_warp(const uint8_t *q, int A, const uint8_t *t, int B, const int8_t *s_mat8, int o, int e,
                           int S, int ei, const int16_t *bm4, int32_t *win, int *amax_out, int *bmax_out) {
    // q[-a], t[-b] for a, b >= 0 walk backwards from the end cell (ei, ej).  The cells of
    // antidiagonal d are those next to the live cells of d-1 (up, left) or of d-2
    // (diagonal).
    const int lane = threadIdx.x & 31;
    const int slack = max(o - e, 0);
    int32_t *WH = win, *WE = win + 3 * WIN, *WF = win + 6 * WIN;
    int lo[3], hi[3];
    if (lane == 0) { WH[0] = 0; WE[0] = NEG; WF[0] = NEG; }
    __syncwarp();
    lo[0] = 0; hi[0] = 0; lo[1] = 1; hi[1] = 0; lo[2] = 1; hi[2] = 0;
    int l1lo = 0, l1hi = 0;          // live range of d-1
    int l2lo = 1, l2hi = 0;          // live range of d-2 (empty)
    int amax = 0, bmax = 0;
    for (int d = 1; d <= A + B; ++d) {
        int clo = 0x7FFFFFFF, chi = -1;
        if (l1lo <= l1hi) { clo = l1lo; chi = l1hi + 1; }
        if (l2lo <= l2hi) { clo = min(clo, l2lo + 1); chi = max(chi, l2hi + 1); }
        if (chi < 0) break;                               // nothing live on d-1 or d-2
        clo = max(max(clo, d - B), 0);
        chi = min(min(chi, A), d);
        if (chi - clo + 1 > WIN) return false;
        const int sc = d % 3, s1 = (d + 2) % 3, s2 = (d + 1) % 3;
        int my_lo = 0x7FFFFFFF, my_hi = -1, my_a = 0, my_b = 0;
        if (clo <= chi) {
            int32_t *Hd = WH + sc * WIN, *Ed = WE + sc * WIN, *Fd = WF + sc * WIN;
            const int32_t *H1 = WH + s1 * WIN, *E1 = WE + s1 * WIN, *F1 = WF + s1 * WIN, *H2 = WH + s2 * WIN;
            const int lo1 = lo[s1], hi1 = hi[s1], lo2 = lo[s2], hi2 = hi[s2];
            for (int a = clo + lane; a <= chi; a += 32) {
                const int b = d - a;
                const int x = a & (WIN - 1), x1 = (a - 1) & (WIN - 1);
                int ev = NEG, fv = NEG, dv = NEG;
                if (b >= 1 && a >= lo1 && a <= hi1) ev = max(H1[x] - o, E1[x] - e);
                if (a >= 1 && a - 1 >= lo1 && a - 1 <= hi1) fv = max(H1[x1] - o, F1[x1] - e);
                if (a >= 1 && b >= 1 && a - 1 >= lo2 && a - 1 <= hi2) {
                    const int hd = H2[x1];
                    if (hd != NEG) dv = hd + s_mat8[q[-(a - 1)] * PASTIS_NSYM + t[-(b - 1)]];
                }
                if (ev < NEG) ev = NEG;
                if (fv < NEG) fv = NEG;
                int h = max(max(dv, fv), ev);
                const int i = ei - a + 1;                 // first forward row of the suffix
                const int thr = S - (i >= 1 ? (int)bm4[(i - 1) >> 1] : 0) - slack;
                if (h < thr) { h = NEG; ev = NEG; fv = NEG; }
                Hd[x] = h; Ed[x] = ev; Fd[x] = fv;
                if (h != NEG) {
                    my_lo = min(my_lo, a);
                    my_hi = max(my_hi, a);
                    if (h == S) { my_a = max(my_a, a); my_b = max(my_b, b); }
                }
            }
            lo[sc] = clo; hi[sc] = chi;
        } else {
            lo[sc] = 1; hi[sc] = 0;
        }
        my_lo = __reduce_min_sync(0xffffffffu, my_lo);
        my_hi = __reduce_max_sync(0xffffffffu, my_hi);
        my_a = __reduce_max_sync(0xffffffffu, my_a);
        my_b = __reduce_max_sync(0xffffffffu, my_b);
        amax = max(amax, my_a);
        bmax = max(bmax, my_b);
        l2lo = l1lo; l2hi = l1hi;
        if (my_hi >= 0) { l1lo = my_lo; l1hi = my_hi; } else { l1lo = 1; l1hi = 0; }
    }
    *amax_out = amax;
    *bmax_out = bmax;
    return true;
}

// Rows per lane: as few stripes as 16 rows per lane allow, then the smallest even row
// count that covers the query in that many stripes.
__device__ __forceinline__ int rows_per_lane(int m) {
    const int ns = max(1, (m + 511) / 512);
    const int per = (m + 32 * ns - 1) / (32 * ns);
    return min(16, max(2, (per + 1) & ~1));
}

__global__ void __launch_bounds__(SW_THREADS, 3) k_sw_score(const uint8_t *qcodes, const int64_t *qoffsets,
                                                         const uint8_t *tcodes, const int64_t *toffsets,
                                                         const pastis_cand *pairs, const int64_t *seg_start,
                                                         int64_t n_seg, const int8_t *gmat, int o, int e,
                                                         int max_s, int prow_cap, char *scratch, size_t warp_bytes,
                                                         int sstride, int *next_seg, sw_score_out *out,
                                                         unsigned long long *cells) {
    // dynamic shared memory: profile [24][prow_cap] int16, then per warp bm4[prow_cap/2] int16
    // and the pass-2 window [9][WIN]
    extern __shared__ __align__(16) int16_t s_prof[];
    __shared__ int s_seg, s_next;
    __shared__ int8_t s_mat8[PASTIS_NSYM * PASTIS_NSYM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * SW_WARPS + warp;
    for (int x = threadIdx.x; x < PASTIS_NSYM * PASTIS_NSYM; x += blockDim.x) s_mat8[x] = gmat[x];
    int16_t *bm4 = s_prof + PASTIS_NSYM * prow_cap + warp * (prow_cap / 2);
    int32_t *win = reinterpret_cast<int32_t *>(s_prof + PASTIS_NSYM * prow_cap + SW_WARPS * (prow_cap / 2)) +
                   warp * 9 * WIN;
    stripe1_cell *my = reinterpret_cast<stripe1_cell *>(scratch + (size_t)gw * warp_bytes);
    unsigned long long my_cells = 0;
    for (;;) {
        if (threadIdx.x == 0) { s_seg = atomicAdd(next_seg, 1); s_next = 0; }
        __syncthreads();
        const int64_t sg = s_seg;
        if (sg >= n_seg) break;
        const int64_t p0 = seg_start[sg], p1 = seg_start[sg + 1];
        const int qi = pairs[p0].i;
        const int64_t qo = qoffsets[qi];
        const int m = (int)(qoffsets[qi + 1] - qo);
        const int lr = rows_per_lane(m);
        const int prow = ((m + 32 * lr - 1) / (32 * lr)) * (32 * lr);
        // query profile: prof[c][i] = M[q_i][c], PAD past the end of the query
        if (prow <= prow_cap) {
            for (int x = threadIdx.x; x < PASTIS_NSYM * prow; x += blockDim.x) {
                const int c = x / prow, i = x - c * prow;
                s_prof[x] = (int16_t)(i < m ? (int)gmat[qcodes[qo + i] * PASTIS_NSYM + c] : PAD_SCORE);
            }
        }
        __syncthreads();
        for (;;) {
            int pk = 0;
            if (lane == 0) pk = atomicAdd(&s_next, 1);
            pk = __shfl_sync(0xffffffffu, pk, 0);
            const int64_t p = p0 + pk;
            if (p >= p1) break;
            const pastis_cand c = pairs[p];
            const int64_t to = toffsets[c.j];
            const int n = (int)(toffsets[c.j + 1] - to);
            sw_score_out r;
            r.score = 0; r.end_i = 0; r.end_j = 0; r.rect_i = 0; r.rect_j = 0; r.big = 0;
            if ((int64_t)max_s * (int64_t)min(m, n) >= 32767 || prow > prow_cap) {
                r.big = 1;                          // left to the int32 carry pass
            } else if (m > 0 && n > 0) {
                int bh, bi, bj;
                const uint8_t *tp = tcodes + to;
#define PASTIS_SW_CASE(L) \
    case L: score_warp<L>(s_prof, prow, tp, m, n, o, e, my, sstride, bm4, &bh, &bi, &bj); break;
                switch (lr) {
                    PASTIS_SW_CASE(2) PASTIS_SW_CASE(4) PASTIS_SW_CASE(6) PASTIS_SW_CASE(8)
                    PASTIS_SW_CASE(10) PASTIS_SW_CASE(12) PASTIS_SW_CASE(14)
                    default: score_warp<16>(s_prof, prow, tp, m, n, o, e, my, sstride, bm4, &bh, &bi, &bj); break;
                }
#undef PASTIS_SW_CASE
                __syncwarp();
                if (bh > 0) {
                    r.score = bh; r.end_i = bi; r.end_j = bj;
                    int amax = 0, bmax = 0;
                    if (bound_warp(qcodes + qo + bi, bi + 1, tp + bj, bj + 1, s_mat8, o, e, bh, bi, bm4, win,
                                   &amax, &bmax) && amax > 0 && bmax > 0) {
                        r.rect_i = bi + 1 - amax;
                        r.rect_j = bj + 1 - bmax;
                    }                                   // else: the whole up-left rectangle
                }
                my_cells += (unsigned long long)m * (unsigned long long)n;
            }
            if (lane == 0) out[p] = r;
        }
        __syncthreads();
    }
    if (lane == 0 && cells && my_cells) atomicAdd(cells, my_cells);
}

// ---------------------------------------------------------------------------------
// pass 3: carries over the rectangle (or the whole matrix for very large scores)
// ---------------------------------------------------------------------------------
constexpr int CR = 8;                  // rows per lane
constexpr int STRIPE3 = 32 * CR;

struct stripe3_cell { int32_t h, f; uint32_t hb, fb, hm, fm; };

__device__ __forceinline__ uint32_t pack_rc(int r, int c) { return ((uint32_t)r << 16) | (uint32_t)c; }

// Carries begin (row << 16 | col, of the first column) and identities << 16 | matched
// columns.  TRACK: also finds the row-major first maximum (for pairs pass 1 skipped);
// otherwise reports the state at (m-1, n-1).
template <bool TRACK>
__device__ void carry_warp(const uint8_t *__restrict__ q, int m, const uint8_t *__restrict__ t, int n,
                           const int *__restrict__ s_mat, int o, int e, stripe3_cell *scratch, int sstride,
                           int *h_out, int *ei_out, int *ej_out, uint32_t *beg_out, uint32_t *im_out) {
    const int lane = threadIdx.x & 31;
    int best = 0, brow = 0x7FFFFFFF, bcol = 0;
    uint32_t bbeg = 0, bim = 0;
    int endh = NEG;
    uint32_t endb = 0, endm = 0;
    const int nstripes = (m + STRIPE3 - 1) / STRIPE3;
    for (int stripe = 0; stripe < nstripes; ++stripe) {
        const int row0 = stripe * STRIPE3 + lane * CR;
        int qoff[CR], Hc[CR], Ec[CR];
        uint32_t HB[CR], EB[CR], HM[CR], EM[CR];
#pragma unroll
        for (int r = 0; r < CR; ++r) {
            const int i = row0 + r;
            qoff[r] = (i < m ? (int)q[i] : PASTIS_NSYM) * 32;
            Hc[r] = 0; Ec[r] = NEG;
            HB[r] = pack_rc(i + 1, 0); EB[r] = 0; HM[r] = 0; EM[r] = 0;
        }
        int dh = 0;
        uint32_t db = pack_rc(row0, 0), dm = 0;
        int out_h = 0, out_f = NEG, out_t = 0;
        uint32_t out_hb = 0, out_fb = 0, out_hm = 0, out_fm = 0;
        const stripe3_cell *in_buf = scratch + (size_t)(stripe & 1) * sstride;
        stripe3_cell *out_buf = scratch + (size_t)((stripe + 1) & 1) * sstride;
        const bool last = stripe + 1 == nstripes;
        for (int s = 0; s < n + 31; ++s) {
            const int j = s - lane;
            int up_h = __shfl_up_sync(0xffffffffu, out_h, 1);
            int up_f = __shfl_up_sync(0xffffffffu, out_f, 1);
            uint32_t up_hb = __shfl_up_sync(0xffffffffu, out_hb, 1);
            uint32_t up_fb = __shfl_up_sync(0xffffffffu, out_fb, 1);
            uint32_t up_hm = __shfl_up_sync(0xffffffffu, out_hm, 1);
            uint32_t up_fm = __shfl_up_sync(0xffffffffu, out_fm, 1);
            int tj = __shfl_up_sync(0xffffffffu, out_t, 1);
            if (lane == 0 && j < n) {
                tj = t[j];
                if (stripe == 0) {
                    up_h = 0; up_f = NEG; up_hb = pack_rc(0, j + 1); up_fb = 0; up_hm = 0; up_fm = 0;
                } else {
                    const stripe3_cell c = in_buf[j];
                    up_h = c.h; up_f = c.f; up_hb = c.hb; up_fb = c.fb; up_hm = c.hm; up_fm = c.fm;
                }
            }
            if (j >= 0 && j < n) {
                int ph = dh;
                uint32_t pb = db, pm = dm;
                int ah = up_h, f = up_f;
                uint32_t ab = up_hb, am = up_hm, fb = up_fb, fm = up_fm;
#pragma unroll
                for (int r = 0; r < CR; ++r) {
                    const int i = row0 + r;
                    const int eo = Hc[r] - o, ex = Ec[r] - e;
                    const bool eop = eo >= ex;
                    const int ev = eop ? eo : ex;
                    const uint32_t evb = eop ? HB[r] : EB[r], evm = eop ? HM[r] : EM[r];
                    const int fo = ah - o, fx = f - e;
                    const bool fop = fo >= fx;
                    f = fop ? fo : fx;
                    fb = fop ? ab : fb;
                    fm = fop ? am : fm;
                    int h = ph + s_mat[qoff[r] + tj];
                    uint32_t hb = pb, hm = pm + ((qoff[r] == tj * 32) ? 0x10001u : 1u);
                    if (f > h) { h = f; hb = fb; hm = fm; }
                    if (ev > h) { h = ev; hb = evb; hm = evm; }
                    if (h <= 0) { h = 0; hb = pack_rc(i + 1, j + 1); hm = 0; }
                    if (TRACK) {
                        if (i < m && (h > best || (h == best && h > 0 && i < brow))) {
                            best = h; brow = i; bcol = j; bbeg = hb; bim = hm;
                        }
                    } else if (i == m - 1 && j == n - 1) {
                        endh = h; endb = hb; endm = hm;
                    }
                    ph = Hc[r]; pb = HB[r]; pm = HM[r];
                    Hc[r] = h; HB[r] = hb; HM[r] = hm;
                    Ec[r] = ev; EB[r] = evb; EM[r] = evm;
                    ah = h; ab = hb; am = hm;
                }
                dh = up_h; db = up_hb; dm = up_hm;
                out_h = ah; out_f = f; out_t = tj;
                out_hb = ab; out_fb = fb; out_hm = am; out_fm = fm;
                if (lane == 31 && !last) out_buf[j] = stripe3_cell{ah, f, ab, fb, am, fm};
            }
        }
        __syncwarp();
    }
    if (TRACK) {
        for (int d = 16; d > 0; d >>= 1) {
            const int ob = __shfl_xor_sync(0xffffffffu, best, d);
            const int orow = __shfl_xor_sync(0xffffffffu, brow, d);
            const int ocol = __shfl_xor_sync(0xffffffffu, bcol, d);
            const uint32_t obb = __shfl_xor_sync(0xffffffffu, bbeg, d);
            const uint32_t obm = __shfl_xor_sync(0xffffffffu, bim, d);
            if (ob > best || (ob == best && (orow < brow || (orow == brow && ocol < bcol)))) {
                best = ob; brow = orow; bcol = ocol; bbeg = obb; bim = obm;
            }
        }
        *h_out = best; *ei_out = brow; *ej_out = bcol; *beg_out = bbeg; *im_out = bim;
    } else {
        for (int d = 16; d > 0; d >>= 1) {
            const int oh = __shfl_xor_sync(0xffffffffu, endh, d);
            const uint32_t ob = __shfl_xor_sync(0xffffffffu, endb, d);
            const uint32_t om = __shfl_xor_sync(0xffffffffu, endm, d);
            if (oh > endh) { endh = oh; endb = ob; endm = om; }
        }
        *h_out = endh; *beg_out = endb; *im_out = endm;
    }
}

// Small rectangles (at most 64 rows): four per warp, each on an 8-lane group with 8
// rows per lane, all groups stepping together (the longest sets the step count) and
// shuffling within their 8 lanes.  Reports the state at each rectangle's last cell.
constexpr int GL = 8;                  // lanes per group
constexpr int GROWS = GL * CR;         // rows per group

__device__ void carry_group(const uint8_t *__restrict__ q, int m, const uint8_t *__restrict__ t, int n,
                            const int *__restrict__ s_mat, int o, int e, int *h_out, uint32_t *beg_out,
                            uint32_t *im_out) {
    const int lane = threadIdx.x & 31, lg = lane & (GL - 1);
    const int row0 = lg * CR;
    int qoff[CR], Hc[CR], Ec[CR];
    uint32_t HB[CR], EB[CR], HM[CR], EM[CR];
#pragma unroll
    for (int r = 0; r < CR; ++r) {
        const int i = row0 + r;
        qoff[r] = (i < m ? (int)q[i] : PASTIS_NSYM) * 32;
        Hc[r] = 0; Ec[r] = NEG;
        HB[r] = pack_rc(i + 1, 0); EB[r] = 0; HM[r] = 0; EM[r] = 0;
    }
    int dh = 0;
    uint32_t db = pack_rc(row0, 0), dm = 0;
    int out_h = 0, out_f = NEG, out_t = 0;
    uint32_t out_hb = 0, out_fb = 0, out_hm = 0, out_fm = 0;
    int endh = NEG;
    uint32_t endb = 0, endm = 0;
    const int nsteps = __reduce_max_sync(0xffffffffu, n > 0 ? n + GL - 1 : 0);
    for (int s = 0; s < nsteps; ++s) {
        const int j = s - lg;
        int up_h = __shfl_up_sync(0xffffffffu, out_h, 1, GL);
        int up_f = __shfl_up_sync(0xffffffffu, out_f, 1, GL);
        uint32_t up_hb = __shfl_up_sync(0xffffffffu, out_hb, 1, GL);
        uint32_t up_fb = __shfl_up_sync(0xffffffffu, out_fb, 1, GL);
        uint32_t up_hm = __shfl_up_sync(0xffffffffu, out_hm, 1, GL);
        uint32_t up_fm = __shfl_up_sync(0xffffffffu, out_fm, 1, GL);
        int tj = __shfl_up_sync(0xffffffffu, out_t, 1, GL);
        if (lg == 0 && j < n) {
            tj = t[j];
            up_h = 0; up_f = NEG; up_hb = pack_rc(0, j + 1); up_fb = 0; up_hm = 0; up_fm = 0;
        }
        if (j >= 0 && j < n) {
            int ph = dh;
            uint32_t pb = db, pm = dm;
            int ah = up_h, f = up_f;
            uint32_t ab = up_hb, am = up_hm, fb = up_fb, fm = up_fm;
#pragma unroll
            for (int r = 0; r < CR; ++r) {
                const int i = row0 + r;
                const int eo = Hc[r] - o, ex = Ec[r] - e;
                const bool eop = eo >= ex;
                const int ev = eop ? eo : ex;
                const uint32_t evb = eop ? HB[r] : EB[r], evm = eop ? HM[r] : EM[r];
                const int fo = ah - o, fx = f - e;
                const bool fop = fo >= fx;
                f = fop ? fo : fx;
                fb = fop ? ab : fb;
                fm = fop ? am : fm;
                int h = ph + s_mat[qoff[r] + tj];
                uint32_t hb = pb, hm = pm + ((qoff[r] == tj * 32) ? 0x10001u : 1u);
                if (f > h) { h = f; hb = fb; hm = fm; }
                if (ev > h) { h = ev; hb = evb; hm = evm; }
                if (h <= 0) { h = 0; hb = pack_rc(i + 1, j + 1); hm = 0; }
                if (i == m - 1 && j == n - 1) { endh = h; endb = hb; endm = hm; }
                ph = Hc[r]; pb = HB[r]; pm = HM[r];
                Hc[r] = h; HB[r] = hb; HM[r] = hm;
                Ec[r] = ev; EB[r] = evb; EM[r] = evm;
                ah = h; ab = hb; am = hm;
            }
            dh = up_h; db = up_hb; dm = up_hm;
            out_h = ah; out_f = f; out_t = tj;
            out_hb = ab; out_fb = fb; out_hm = am; out_fm = fm;
        }
    }
    for (int d = GL / 2; d > 0; d >>= 1) {
        const int oh = __shfl_xor_sync(0xffffffffu, endh, d, GL);
        const uint32_t ob = __shfl_xor_sync(0xffffffffu, endb, d, GL);
        const uint32_t om = __shfl_xor_sync(0xffffffffu, endm, d, GL);
        if (oh > endh) { endh = oh; endb = ob; endm = om; }
    }
    *h_out = endh; *beg_out = endb; *im_out = endm;
}

__device__ void finish_record(pastis_aln &rec, int S, int ei, int ej, int qb, int tb, int ident, int M, int lq,
                              int lt, int ani, int cov) {
    rec.score = S;
    rec.qb = (uint16_t)qb; rec.qe = (uint16_t)(ei + 1); rec.tb = (uint16_t)tb; rec.te = (uint16_t)(ej + 1);
    rec.ident = (uint16_t)ident;
    rec.cols = (uint16_t)((ei + 1 - qb) + (ej + 1 - tb) - M);
    const int span = lq <= lt ? ei + 1 - qb : ej + 1 - tb;
    const int L = lq <= lt ? lq : lt;
    rec.passes = (rec.cols > 0 && 100 * ident >= ani * (int)rec.cols && 100 * span >= cov * L) ? 1 : 0;
}

__global__ void __launch_bounds__(SW_THREADS) k_sw_carry(const uint8_t *qcodes, const int64_t *qoffsets,
                                                         const uint8_t *tcodes, const int64_t *toffsets,
                                                         const pastis_cand *pairs, int64_t n_pairs,
                                                         const int8_t *gmat, int o, int e, int ani, int cov,
                                                         stripe3_cell *scratch, int sstride, int *next_pair,
                                                         const sw_score_out *res, pastis_aln *out, int *err,
                                                         unsigned long long *cells) {
    __shared__ int s_mat[(PASTIS_NSYM + 1) * 32];
    for (int x = threadIdx.x; x < (PASTIS_NSYM + 1) * 32; x += blockDim.x) {
        const int a = x / 32, b = x % 32;
        s_mat[x] = (a < PASTIS_NSYM && b < PASTIS_NSYM) ? (int)gmat[a * PASTIS_NSYM + b] : PAD_SCORE;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, grp = lane / GL, lg = lane & (GL - 1);
    const int gw = blockIdx.x * SW_WARPS + (threadIdx.x >> 5);
    stripe3_cell *my = scratch + (size_t)gw * 2 * sstride;
    unsigned long long my_cells = 0;
    for (;;) {
        int p0 = 0;
        if (lane == 0) p0 = atomicAdd(next_pair, 32 / GL);
        p0 = __shfl_sync(0xffffffffu, p0, 0);
        if (p0 >= n_pairs) break;
        // the four pairs of this warp: small rectangles go to the groups together
        const int64_t pg = p0 + grp;
        int gm = 0, gn = 0;
        const uint8_t *gq = qcodes, *gt = tcodes;
        sw_score_out g1;
        g1.score = 0; g1.big = 0; g1.end_i = g1.end_j = g1.rect_i = g1.rect_j = 0;
        if (pg < n_pairs) {
            g1 = res[pg];
            if (!g1.big && g1.score > 0 && g1.end_i + 1 - g1.rect_i <= GROWS) {
                const pastis_cand c = pairs[pg];
                gm = g1.end_i + 1 - g1.rect_i;
                gn = g1.end_j + 1 - g1.rect_j;
                gq = qcodes + qoffsets[c.i] + g1.rect_i;
                gt = tcodes + toffsets[c.j] + g1.rect_j;
            }
        }
        int gh;
        uint32_t gb, gim;
        carry_group(gq, gm, gt, gn, s_mat, o, e, &gh, &gb, &gim);
        if (lg == 0 && pg < n_pairs && gm > 0) {
            const pastis_cand c = pairs[pg];
            const int lq = (int)(qoffsets[c.i + 1] - qoffsets[c.i]), lt = (int)(toffsets[c.j + 1] - toffsets[c.j]);
            if (gh != g1.score) atomicExch(err, 1);
            pastis_aln rec;
            rec.seed_used = 0; rec.passes = 0; rec.reserved = 0;
            finish_record(rec, g1.score, g1.end_i, g1.end_j, g1.rect_i + (int)(gb >> 16), g1.rect_j + (int)(gb & 0xFFFF),
                          (int)(gim >> 16), (int)(gim & 0xFFFF), lq, lt, ani, cov);
            out[pg] = rec;
        }
        // the others, one warp each
        for (int k = 0; k < 32 / GL; ++k) {
            const int64_t p = p0 + k;
            if (p >= n_pairs) break;
            const sw_score_out r1 = res[p];
            const bool small = !r1.big && r1.score > 0 && r1.end_i + 1 - r1.rect_i <= GROWS;
            if (small) continue;
            const pastis_cand c = pairs[p];
            const int64_t qo = qoffsets[c.i], to = toffsets[c.j];
            const int lq = (int)(qoffsets[c.i + 1] - qo), lt = (int)(toffsets[c.j + 1] - to);
            pastis_aln rec;
            rec.score = 0; rec.qb = rec.qe = rec.tb = rec.te = 0; rec.ident = rec.cols = 0;
            rec.seed_used = 0; rec.passes = 0; rec.reserved = 0;
            if (r1.big) {
                if (lq > 0 && lt > 0) {
                    int h, bi, bj;
                    uint32_t beg, im;
                    carry_warp<true>(qcodes + qo, lq, tcodes + to, lt, s_mat, o, e, my, sstride, &h, &bi, &bj, &beg, &im);
                    if (h > 0)
                        finish_record(rec, h, bi, bj, (int)(beg >> 16), (int)(beg & 0xFFFF), (int)(im >> 16),
                                      (int)(im & 0xFFFF), lq, lt, ani, cov);
                    if (lane == 0) my_cells += (unsigned long long)lq * lt;
                }
            } else if (r1.score > 0) {
                const int ri = r1.rect_i, rj = r1.rect_j;
                int h, dummy_i, dummy_j;
                uint32_t beg, im;
                carry_warp<false>(qcodes + qo + ri, r1.end_i + 1 - ri, tcodes + to + rj, r1.end_j + 1 - rj, s_mat, o,
                                  e, my, sstride, &h, &dummy_i, &dummy_j, &beg, &im);
                if (h != r1.score && lane == 0) atomicExch(err, 1);
                finish_record(rec, r1.score, r1.end_i, r1.end_j, ri + (int)(beg >> 16), rj + (int)(beg & 0xFFFF),
                              (int)(im >> 16), (int)(im & 0xFFFF), lq, lt, ani, cov);
            }
            if (lane == 0) out[p] = rec;
        }
    }
    if (lane == 0 && cells && my_cells) atomicAdd(cells, my_cells);
}

}  // namespace

// Host side of the Smith-Waterman path (called by pastis_align_pairs after validation).
pastis_status sw_align(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets, const uint8_t *d_tcodes,
                       const int64_t *d_toffsets, const pastis_cand *d_pairs,
                       int64_t n_pairs, const pastis_params *p, const int8_t *dmat, int *flags, int lmax,
                       pastis_aln *d_out, int64_t *d_cells) {
    cudaStream_t st = ctx->stream;
    int max_s = 0;
    for (int x = 0; x < PASTIS_NSYM * PASTIS_NSYM; ++x) max_s = std::max(max_s, (int)p->matrix[x]);
    // segments of pairs sharing a query
    uint32_t *sflags;
    PASTIS_WS(sflags, ctx, WS_ALN_ORDER, sizeof(uint32_t) * (2 * (size_t)n_pairs + 2) + sizeof(int64_t) * (n_pairs + 2) + 16);
    uint32_t *soff = sflags + n_pairs + 1;
    int64_t *seg_start = (int64_t *)(((uintptr_t)(soff + n_pairs + 1) + 7) & ~(uintptr_t)7);
    k_seg_flags<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(d_pairs, n_pairs, sflags);
    PASTIS_LAUNCHED(ctx);
    pastis_status s = exclusive_scan_u32(ctx, sflags, soff, n_pairs);
    if (s != PASTIS_OK) return s;
    k_seg_starts<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(sflags, soff, n_pairs, seg_start);
    PASTIS_LAUNCHED(ctx);
    uint32_t h_nseg = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&h_nseg, soff + n_pairs, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));

    sw_score_out *res;
    PASTIS_WS(res, ctx, WS_ALN_PASS1, sizeof(sw_score_out) * (size_t)n_pairs);
    // pass 1+2: profile rows up to the longest query (in whole stripes), within shared memory
    int prow_cap = ((lmax + STRIPE1 - 1) / STRIPE1) * STRIPE1;
    if (prow_cap < STRIPE1) prow_cap = STRIPE1;
    auto shm_for = [](int pc) {
        return (size_t)PASTIS_NSYM * pc * 2 + (size_t)SW_WARPS * (pc / 2) * 2 + (size_t)SW_WARPS * 9 * WIN * 4;
    };
    while (prow_cap > STRIPE1 && shm_for(prow_cap) + 1024 > ctx->smem_optin) prow_cap -= STRIPE1;
    const size_t shm1 = shm_for(prow_cap);
    cudaFuncSetAttribute(k_sw_score, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm1);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sw_score, SW_THREADS, shm1);
    if (per_sm < 1) per_sm = 1;
    const int blocks1 = ctx->sm_count * per_sm;
    const int sstride = lmax + 1;
    const size_t warp_bytes = (sizeof(stripe1_cell) * 2 * (size_t)sstride + 255) & ~(size_t)255;
    const size_t scr1 = warp_bytes * (size_t)blocks1 * SW_WARPS;
    const int blocks3 = ctx->sm_count * 2;
    const size_t scr3 = sizeof(stripe3_cell) * (size_t)blocks3 * SW_WARPS * 2 * sstride;
    void *scratch;
    PASTIS_WS(scratch, ctx, WS_ALN_SCRATCH, std::max(scr1, scr3));
    prof_begin(ctx, "sw_pass1");
    k_sw_score<<<blocks1, SW_THREADS, shm1, st>>>(d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs, seg_start,
                                                  (int64_t)h_nseg, dmat,
                                                  p->gap_open, p->gap_extend, max_s, prow_cap, (char *)scratch,
                                                  warp_bytes, sstride, flags + 1, res, (unsigned long long *)d_cells);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    prof_begin(ctx, "sw_pass3");
    k_sw_carry<<<blocks3, SW_THREADS, 0, st>>>(d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs, n_pairs, dmat,
                                               p->gap_open,
                                               p->gap_extend, p->ani_min_pct, p->cov_min_pct,
                                               (stripe3_cell *)scratch, sstride, flags + 8, res, d_out, flags,
                                               (unsigned long long *)d_cells);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    return PASTIS_OK;
}
