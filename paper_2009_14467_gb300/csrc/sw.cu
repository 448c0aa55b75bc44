// a8: Smith-Waterman of candidate pairs (Sec. IV-E, Sec. VI), three passes.
//
// Recurrences (a gap of length L costs open + (L-1)*extend):
//   E(i,j) = max(H(i,j-1) - o, E(i,j-1) - e)     F(i,j) = max(H(i-1,j) - o, F(i-1,j) - e)
//   H(i,j) = max(0, H(i-1,j-1) + s(q_i, t_j), F(i,j), E(i,j))
// Reported: the score S, the end = the first maximum in row-major order, and the
// alignment a traceback from the end selects when it prefers the diagonal, then F,
// then E, and a gap open over an extension (its begin, identities, columns).
//
// Pass 1 (the whole matrix, every pair): score and end only.  A warp takes two pairs
//   that share the query (candidate lists are grouped by i; within a run of pairs of
//   one query they are taken in order of target length, so the two matrices match)
//   and holds them in the two 16-bit halves of each register, so one 16x2 maximum or
//   one 32-bit add advances both.  Lane l owns up to 16 consecutive query rows and at
//   step s computes column j = s - l, taking H/F of the row above from lane l-1
//   (__shfl_up_sync).  Scores come from a biased query profile in shared memory
//   (one byte per [target residue][query row]) shared by every warp of the CTA.  Each row
//   keeps a key (H << 16 | 65535 - j) of its first maximum; the end is the first row
//   with the best score, at that row's first maximum: the row-major first maximum.
//   Pass 1 also stores, per pair of query rows, the largest H it met there.
//   Queries longer than one stripe of 32 * 16 rows go in stripes whose last row is
//   handed on through a per-warp buffer.
// Pass 2 (its own kernel, one warp per pair; a band around the path): an anchored DP
//   over the reversed prefixes from the end (ei, ej), row by row with up to 64 columns
//   per row (two per lane; antidiagonal by antidiagonal when a row needs more or the
//   gap costs have o < e).  A suffix of the traced path starting on row i scores S minus
//   the forward value before it, which is at most the largest H pass 1 met on row
//   i-1's pair of rows; cells below that threshold die, the path's suffixes all
//   survive, and the cells reaching S bound the begin.  Their extent gives a rectangle
//   that contains the whole traced path.
// Pass 3 (that rectangle): the DP again with zero boundaries; each state carries its
//   begin cell and (identities << 16 | matched columns) along the predecessor a
//   traceback would take.  Inside a rectangle holding the path, the path's cells keep
//   their values and every choice along it is the same, so the carry at the end cell
//   is the traceback's.  cols = span_q + span_t - matched.
// Pairs whose scores could reach SCORE_MAX (max score * shorter length), gap opens
// above GAP_MAX, and queries longer than the shared-memory profile take pass 3 over the
// whole matrix with the end tracked there instead (int32).
// Captured launch sequences (alignment plans) pass device-side counts: each kernel then
// reads its pair or segment count from device memory and does nothing when the input
// checks flagged the batch.
#include <algorithm>

#include "internal.cuh"

namespace {

constexpr int NEG = -1000000000;
constexpr int SW_THREADS = 256;
constexpr int SW_WARPS = SW_THREADS / 32;
constexpr int STRIPE1 = 512;               // rows per stripe in pass 1 at 16 rows per lane
constexpr int PAD_SCORE = -30000;
constexpr int SEG_MAX = 128;               // pairs per scheduling segment

struct sw_score_out {                      // pass 1 result per pair
    int32_t score;
    int32_t end_i, end_j;
    int32_t rect_i, rect_j;                // pass 2: start of the bounding rectangle
    int32_t big;                           // scores may not fit the pass-1 key
};

// The filter-only mode (PASTIS_SW_FILTERED): the traced path lies in the rectangle
// [rect_i, end_i] x [rect_j, end_j] (the whole up-left rectangle before pass 2 narrows
// it), so its span on the shorter sequence (i on equal lengths) is at most the
// rectangle's extent there.  An extent below the coverage bound means the pair cannot
// pass the filter, and its begin and carried statistics are never needed.
__device__ __forceinline__ bool cannot_cover(const sw_score_out &r, int lq, int lt, int cov) {
    const int ext = lq <= lt ? r.end_i + 1 - r.rect_i : r.end_j + 1 - r.rect_j;
    return 100 * ext < cov * min(lq, lt);
}

// ---------------------------------------------------------------------------------
// segments: runs of pairs with the same query, at most SEG_MAX long
// ---------------------------------------------------------------------------------
// dn (captured launches): the pair count in device memory, n the capacity; 0 past it.
__global__ void k_seg_flags(const pastis_cand *pairs, int64_t n, uint32_t *flags, const int64_t *dn) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t m = dn ? *dn : n;
    flags[p] = p < m && (p == 0 || (p % SEG_MAX) == 0 || pairs[p].i != pairs[p - 1].i) ? 1u : 0u;
}

__global__ void k_seg_starts(const uint32_t *flags, const uint32_t *off, int64_t n, int64_t *seg_start,
                             const int64_t *dn) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t m = dn ? *dn : n;
    if (p < m && flags[p]) seg_start[off[p]] = p;
    if (p == m - 1) seg_start[off[p] + flags[p]] = m;
}

// ---------------------------------------------------------------------------------
// pass 1: two pairs per warp, one in each 16-bit half of every register
// ---------------------------------------------------------------------------------
// Every state is a signed 16-bit half: H >= 0, E and F >= -o (a gap is at least as good
// as opening it from H >= 0), and nothing exceeds the best score plus one substitution,
// so with no score reaching SCORE_MAX all values fit.  Per-half adds wrap within their
// half, and the 16x2 maximum instructions (max(a + b, c) and max(a, b, c, 0)) advance
// both pairs at once.  The profile stores score + o in a signed byte, so o <= GAP_MAX.
constexpr int GAP_MAX = 64;
constexpr int SCORE_MAX = 32000;
constexpr uint32_t P2 = 0x00010001u;
constexpr int NRES = PASTIS_NSYM + 1;      // profile rows: the residues, then the pad residue
constexpr int PAD_RES = PASTIS_NSYM;       // stands for target columns past the shorter target

// prmt with the sign-replicate bit of its selector (bytes below 0x80 become 0x00)
__device__ __forceinline__ uint32_t prmt_sx(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}
// a * b + c as a multiply-add (b is the run-time 1 the kernel receives, so the add goes
// to the multiply-add pipe and leaves the integer ALU pipe to the maxima)
__device__ __forceinline__ uint32_t madd(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

struct end_cell { int h, i, j; };

// Rows per lane: as few stripes as 16 rows per lane allow, plus `extra` stripes (the
// layout the tuner picked for the query's length bin), then the smallest row count
// (at least 2) that covers the query in that many stripes.  More stripes pad fewer rows
// but sweep the target more often; the layout changes no result.
__device__ __forceinline__ int rows_per_lane(int m, int extra) {
    const int ns = max(1, (m + 511) / 512) + extra;
    const int per = (m + 32 * ns - 1) / (32 * ns);
    return min(16, max(2, per));
}

// The profile holds one signed byte per (target residue, query row): score + o, and
// o - 64 (the lowest score) for the pad residue and past the query.  Rows are laid out
// per stripe and lane in 16-byte slots (slot of lane l in stripe st at st * 512 + l * 16,
// row r of the lane at +r), so a lane reads its rows of one column with one 16-byte load.
constexpr int SLOT = 16;
constexpr int STRIPE_BYTES = 32 * SLOT;

// One column of a lane's LR rows for both pairs.  Ho = H - o is kept per row (it feeds
// E, F and the keys), so the diagonal term is Ho(i-1, j-1) + (score + o).  The key of a
// row keeps (Ho << 16 | 65535 - j) of its best column as a signed word: the largest Ho,
// then the first column, i.e. the first maximum of that row.  Pair A's key is
// Ho * 2^16 + jt (pair B's half leaves the word), pair B's is (Ho & 0xFFFF0000) | jt.
template <int LR>
__device__ __forceinline__ void column2(const uint8_t *__restrict__ pa, const uint8_t *__restrict__ pb,
                                        uint32_t (&Ho)[LR], uint32_t (&E)[LR], uint32_t (&kA)[LR],
                                        uint32_t (&kB)[LR], uint32_t hdiag, uint32_t &f, uint32_t &hup, uint32_t jt,
                                        uint32_t sh16, uint32_t OP, uint32_t nEP) {
    const uint4 x = *reinterpret_cast<const uint4 *>(pa), y = *reinterpret_cast<const uint4 *>(pb);
    const uint32_t wa[4] = {x.x, x.y, x.z, x.w}, wb[4] = {y.x, y.y, y.z, y.w};
    // byte r of the two words into the low and high halves, sign-extended
    constexpr uint32_t SEL[4] = {0xc480u, 0xd591u, 0xe6a2u, 0xf7b3u};
#pragma unroll
    for (int r = 0; r < LR; ++r) {
        const uint32_t s = prmt_sx(wa[r >> 2], wb[r >> 2], SEL[r & 3]);
        const uint32_t d = __vadd2(hdiag, s);                 // H(i-1, j-1) + score
        E[r] = __viaddmax_s16x2(E[r], nEP, Ho[r]);            // E(i, j) = max(E(i, j-1) - e, H(i, j-1) - o)
        f = __viaddmax_s16x2(f, nEP, hup);                    // F(i, j) = max(F(i-1, j) - e, H(i-1, j) - o)
        const uint32_t h = __vimax3_s16x2_relu(d, E[r], f);   // H = max(0, diagonal, E, F)
        hdiag = Ho[r];
        Ho[r] = __vsub2(h, OP);
        hup = Ho[r];
        kA[r] = (uint32_t)max((int)kA[r], (int)madd(Ho[r], sh16, jt));
        kB[r] = (uint32_t)max((int)kB[r], (int)((Ho[r] & 0xFFFF0000u) | jt));
    }
}

// The registers a pass-1 stripe sweep carries from column to column, and the values
// that stay fixed over the sweep.
template <int LR>
struct pass1_state {
    uint32_t (&Ho)[LR], (&E)[LR], (&kA)[LR], (&kB)[LR];
    uint32_t &hd, &out_h, &out_f, &out_t, &twin, &tnext;
};
struct pass1_consts {
    const uint8_t *pr;
    int prow8;
    const uint8_t *tA;
    int nA;
    const uint8_t *tB;
    int nB, n, lane;
    bool first_stripe, hand_on;
    uint32_t INIT, sh16, OP, nEP;
    const uint2 *in_buf;
    uint2 *out_buf;
};

// The target window at step s (a multiple of 32): columns [s, s + 32) move to twin,
// and lane k loads column s + 32 + k of both targets into tnext.
template <int LR>
__device__ __forceinline__ void pass1_window(const int s, const pass1_consts &c, pass1_state<LR> &st) {
    st.twin = st.tnext;
    const int x = s + 32 + c.lane;
    st.tnext = (x < c.nA ? (uint32_t)c.tA[x] : (uint32_t)PAD_RES) |
               ((x < c.nB ? (uint32_t)c.tB[x] : (uint32_t)PAD_RES) << 16);
}

// One step s of the wavefront: lane l computes column j = s - l of its rows.  CHECKED
// tests that j is a column (the ramps); `window` = false when the caller loads the
// target windows itself.
template <int LR, bool CHECKED>
__device__ __forceinline__ void pass1_step(const int s, const pass1_consts &c, pass1_state<LR> &st,
                                           const bool window = true) {
    const int lane = c.lane, j = s - lane;
    if (window && s > 0 && (s & 31) == 0) pass1_window<LR>(s, c, st);
    const uint32_t tw = __shfl_sync(0xffffffffu, st.twin, s & 31);
    uint32_t hu = __shfl_up_sync(0xffffffffu, st.out_h, 1);
    uint32_t fu = __shfl_up_sync(0xffffffffu, st.out_f, 1);
    uint32_t tt = __shfl_up_sync(0xffffffffu, st.out_t, 1);
    if (lane == 0) {
        tt = tw;
        if (c.first_stripe) { hu = c.INIT; fu = c.INIT; }
        else if (!CHECKED || j < c.n) { const uint2 v = c.in_buf[j]; hu = v.x; fu = v.y; }
    }
    if (!CHECKED || (j >= 0 && j < c.n)) {
        uint32_t f = fu, hup = hu;
        column2<LR>(c.pr + (int)(tt & 0xFFFFu) * c.prow8, c.pr + (int)(tt >> 16) * c.prow8, st.Ho, st.E, st.kA,
                    st.kB, st.hd, f, hup, 65535u - (uint32_t)j, c.sh16, c.OP, c.nEP);
        st.hd = hu;
        st.out_h = hup; st.out_f = f; st.out_t = tt;
        if (lane == 31 && c.hand_on) c.out_buf[j] = make_uint2(hup, f);
    }
}

// Pass 1 over the whole matrix of two pairs with the same query: pair A (target tA,
// nA columns) in the low halves, pair B in the high halves.  Lane l owns LR
// consecutive query rows and at step s does column j = s - l, taking the row above from
// lane l-1; a stripe is 32 * LR rows, its last row handed on through buf.  Columns
// past the shorter target use the pad residue, which scores -64 against every row: a
// cell there stays below the best score of its own pair, so it never becomes the end.
// Lane 0 takes the target residues from a window of 32 columns that the warp loads one
// window ahead.  Returns each pair's best score and its first maximum in row-major
// order, and writes bm[g] = the largest H on rows 2g and 2g+1 (pass 2's bound).
template <int LR>
__device__ void score_pair(const uint8_t *__restrict__ prof, int prow8, const uint8_t *__restrict__ tA, int nA,
                           const uint8_t *__restrict__ tB, int nB, int m, int o, int e, uint32_t one, uint2 *buf,
                           int sstride, int16_t *bmA, int16_t *bmB, end_cell *ra, end_cell *rb) {
    constexpr int STRIPE = 32 * LR;
    const int lane = threadIdx.x & 31;
    const int n = max(nA, nB);
    const uint32_t INIT = ((uint32_t)(-o) & 0xFFFFu) * P2;  // -o in both halves
    const uint32_t OP = (uint32_t)o * P2, nEP = ((uint32_t)(-e) & 0xFFFFu) * P2;
    const uint32_t sh16 = one << 16;                        // 2^16 at run time (keeps the multiply-add)
    int bA = -1, iA = 0, jA = 0, bB = -1, iB = 0, jB = 0;
    const int nstripes = (m + STRIPE - 1) / STRIPE;
    for (int stripe = 0; stripe < nstripes; ++stripe) {
        const int row0 = stripe * STRIPE + lane * LR;
        uint32_t Ho[LR], E[LR], kA[LR], kB[LR];
#pragma unroll
        for (int r = 0; r < LR; ++r) { Ho[r] = INIT; E[r] = INIT; kA[r] = 0x80000000u; kB[r] = 0x80000000u; }
        uint32_t hd = INIT;                                 // Ho(row0 - 1, j - 1)
        uint32_t out_h = INIT, out_f = INIT, out_t = 0;
        const uint2 *in_buf = buf + (size_t)(stripe & 1) * sstride;
        uint2 *out_buf = buf + (size_t)((stripe + 1) & 1) * sstride;
        const bool last = stripe + 1 == nstripes;
        const uint8_t *pr = prof + stripe * STRIPE_BYTES + lane * SLOT;
        // target residues of columns [w, w + 32) (lane k holds column w + k), and the next window
        uint32_t twin = (lane < nA ? (uint32_t)tA[lane] : (uint32_t)PAD_RES) |
                        ((lane < nB ? (uint32_t)tB[lane] : (uint32_t)PAD_RES) << 16);
        uint32_t tnext = (32 + lane < nA ? (uint32_t)tA[32 + lane] : (uint32_t)PAD_RES) |
                         ((32 + lane < nB ? (uint32_t)tB[32 + lane] : (uint32_t)PAD_RES) << 16);
        // Steps [0, 31) and [n, n + 31) are the wavefront's ramps, where some lanes have
        // no column; in [31, n) every lane has one, so those steps skip the range tests
        // and run in runs that end at the next 32-column window boundary, the window
        // loaded once per run instead of tested at every step (measured on the 100k
        // step: pass 1 -7% against one loop with the tests in every step).
        pass1_state<LR> st{Ho, E, kA, kB, hd, out_h, out_f, out_t, twin, tnext};
        const pass1_consts pc{pr, prow8, tA, nA, tB, nB, n, lane, stripe == 0, !last, INIT, sh16, OP, nEP,
                              in_buf, out_buf};
        int s = 0;
        for (const int s_up = min(31, n + 31); s < s_up; ++s) pass1_step<LR, true>(s, pc, st);
        while (s < n) {
            if ((s & 31) == 0) pass1_window<LR>(s, pc, st);
            const int ce = min(n, (s | 31) + 1);          // up to the next window boundary
#pragma unroll 2
            for (; s < ce; ++s) pass1_step<LR, false>(s, pc, st, false);
        }
        for (; s < n + 31; ++s) pass1_step<LR, true>(s, pc, st);
        // this lane's rows: first maximum per pair, and the row-pair bounds.  With LR odd
        // every other lane starts on an odd row, so the pair (2g, 2g+1) may straddle two
        // lanes: the lane holding row 2g takes row 2g+1's maximum from the next lane.  A
        // stripe (32 LR rows) starts on an even row, so no pair straddles two stripes.
        const int nxa = __shfl_down_sync(0xffffffffu, ((int)kA[0] >> 16) + o, 1);
        const int nxb = __shfl_down_sync(0xffffffffu, ((int)kB[0] >> 16) + o, 1);
#pragma unroll
        for (int r = 0; r < LR; ++r) {
            const int xa0 = ((int)kA[r] >> 16) + o, xb0 = ((int)kB[r] >> 16) + o;
            const int xa1 = r + 1 < LR ? ((int)kA[(r + 1) % LR] >> 16) + o : nxa;
            const int xb1 = r + 1 < LR ? ((int)kB[(r + 1) % LR] >> 16) + o : nxb;
            const int i = row0 + r;
            if (i < m) {
                if ((i & 1) == 0) {
                    bmA[i >> 1] = (int16_t)max(xa0, xa1);
                    bmB[i >> 1] = (int16_t)max(xb0, xb1);
                }
                if (xa0 > bA) { bA = xa0; iA = i; jA = 65535 - (int)(kA[r] & 0xFFFFu); }
                if (xb0 > bB) { bB = xb0; iB = i; jB = 65535 - (int)(kB[r] & 0xFFFFu); }
            }
        }
        __syncwarp();
    }
    // across the warp: the largest score, then the smallest row (rows are unique per lane)
    const int SA = __reduce_max_sync(0xffffffffu, bA), SB = __reduce_max_sync(0xffffffffu, bB);
    const int eiA = (int)__reduce_min_sync(0xffffffffu, bA == SA ? (unsigned)iA : 0xFFFFFFFFu);
    const int eiB = (int)__reduce_min_sync(0xffffffffu, bB == SB ? (unsigned)iB : 0xFFFFFFFFu);
    const unsigned wa = __ballot_sync(0xffffffffu, bA == SA && iA == eiA);
    const unsigned wb = __ballot_sync(0xffffffffu, bB == SB && iB == eiB);
    ra->h = SA; ra->i = eiA; ra->j = __shfl_sync(0xffffffffu, jA, __ffs(wa) - 1);
    rb->h = SB; rb->i = eiB; rb->j = __shfl_sync(0xffffffffu, jB, __ffs(wb) - 1);
}

// ---------------------------------------------------------------------------------
// pass 2: bounding rectangle of the traced path, by an anchored DP over the reversed
// prefixes in which cells below a bound die
// ---------------------------------------------------------------------------------
// The suffix of the traced path that starts on forward row i scores S minus the
// forward value of the path state before it, which sits on row i-1; that value is at
// most bm[(i-1)/2], the largest H pass 1 saw on that pair of rows.  When the split
// falls inside a gap run, the reverse DP charges the suffix's part of the run an open
// instead of an extension, so its reverse value can be lower by o - e.  A reverse cell
// whose first row is i therefore dies below S - bm[(i-1)/2] - (o - e) (bm = 0 above
// row 0); every suffix of the path meets the bound, so the path survives, and the
// cells reaching S bound its begin.
// The band of an antidiagonal (a = rows back from the end, b = d - a columns back) is
// held two cells per lane, index k in lane k % 32 of chunk k / 32; the neighbours on
// the two antidiagonals before come by shuffles.  A live band wider than BAND cells
// returns false and the caller keeps the whole up-left rectangle.
constexpr int BAND = 64;

// The value the previous antidiagonal holds at band index idx (NEG outside the band).
// `wide` is the same on every lane.
__device__ __forceinline__ int band_get(const int (&X)[2], int idx, bool wide) {
    const int v0 = __shfl_sync(0xffffffffu, X[0], idx & 31);
    int v = v0;
    if (wide) {
        const int v1 = __shfl_sync(0xffffffffu, X[1], idx & 31);
        v = idx >= 32 ? v1 : v0;
    }
    return (unsigned)idx < (wide ? 64u : 32u) ? v : NEG;
}

__device__ __noinline__ bool band_walk(const uint8_t *__restrict__ q, const uint8_t *__restrict__ t, const int *s_mat, int o,
                          int e, int S, int ei, int ej, const int16_t *__restrict__ bm, int *amax_out,
                          int *bmax_out) {
    const int lane = threadIdx.x & 31;
    const int A = ei + 1, B = ej + 1;
    const int slack = max(o - e, 0);
    int H1[2] = {lane == 0 ? 0 : NEG, NEG}, E1[2] = {NEG, NEG}, F1[2] = {NEG, NEG};   // d-1 (d = 0: the end)
    int H2[2] = {NEG, NEG};                                                          // d-2
    int w1 = 0, W1 = 1, w2 = 0, W2 = 0;            // band start and computed width of d-1, d-2
    int l1lo = 0, l1hi = 0, l2lo = 1, l2hi = 0;    // live ranges of a on d-1, d-2
    int amax = 0, bmax = 0;
    for (int d = 1; d <= A + B; ++d) {
        int clo = 0x7FFFFFFF, chi = -1;
        if (l1lo <= l1hi) { clo = l1lo; chi = l1hi + 1; }
        if (l2lo <= l2hi) { clo = min(clo, l2lo + 1); chi = max(chi, l2hi + 1); }
        if (chi < 0) break;                        // nothing live on d-1 or d-2
        clo = max(max(clo, d - B), 0);
        chi = min(min(chi, A), d);
        const int W = max(chi - clo + 1, 0);
        if (W > BAND) return false;
        const bool wide = W > 32 || W1 > 32 || W2 > 32;
        int h[2] = {NEG, NEG}, ev[2] = {NEG, NEG}, fv[2] = {NEG, NEG};
        unsigned live[2] = {0u, 0u};
        int ta = 0, tb = 0;                        // this lane's largest (a, b) reaching S
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (c == 1 && !wide) break;
            const int a = clo + 32 * c + lane, b = d - a;
            const int sa = a - w1, su = a - 1 - w1, s2 = a - 1 - w2;
            const int h1a = band_get(H1, sa, wide), e1a = band_get(E1, sa, wide);
            const int h1u = band_get(H1, su, wide), f1u = band_get(F1, su, wide);
            const int h2 = band_get(H2, s2, wide);
            if (a <= chi) {
                if (b >= 1) ev[c] = max(max(h1a - o, e1a - e), NEG);
                if (a >= 1) fv[c] = max(max(h1u - o, f1u - e), NEG);
                int dv = NEG;
                if (a >= 1 && b >= 1 && h2 != NEG)
                    dv = h2 + s_mat[(int)q[ei - (a - 1)] * PASTIS_NSYM + (int)t[ej - (b - 1)]];
                int hh = max(max(dv, ev[c]), fv[c]);
                const int i = ei - a + 1;          // first forward row of the suffix
                const int thr = S - (i >= 1 ? (int)bm[(i - 1) >> 1] : 0) - slack;
                if (hh < thr) { hh = NEG; ev[c] = NEG; fv[c] = NEG; }
                h[c] = hh;
                if (hh == S) { ta = a; tb = max(tb, b); }
            }
            live[c] = __ballot_sync(0xffffffffu, h[c] != NEG);
        }
        if (__any_sync(0xffffffffu, ta > 0 || tb > 0)) {
            amax = max(amax, __reduce_max_sync(0xffffffffu, ta));
            bmax = max(bmax, __reduce_max_sync(0xffffffffu, tb));
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) { H2[c] = H1[c]; H1[c] = h[c]; E1[c] = ev[c]; F1[c] = fv[c]; }
        w2 = w1; W2 = W1; w1 = clo; W1 = W;
        l2lo = l1lo; l2hi = l1hi;
        if (live[0] | live[1]) {
            l1lo = clo + (live[0] ? __ffs(live[0]) - 1 : 32 + __ffs(live[1]) - 1);
            l1hi = clo + (live[1] ? 63 - __clz(live[1]) : 31 - __clz(live[0]));
        } else {
            l1lo = 1; l1hi = 0;
        }
    }
    *amax_out = amax;
    *bmax_out = bmax;
    return true;
}

// The value the previous row holds at window index idx (two columns per lane; NEG
// outside the window).  `wide` (the previous row used its second chunk) is the same
// on every lane.
__device__ __forceinline__ int row_get(const int (&X)[2], int idx, bool wide) {
    const int v0 = __shfl_sync(0xffffffffu, X[0], idx & 31);
    int v = v0;
    if (wide) {
        const int v1 = __shfl_sync(0xffffffffu, X[1], idx & 31);
        v = idx >= 32 ? v1 : v0;
    }
    return (unsigned)idx < (wide ? 64u : 32u) ? v : NEG;
}

// The same reverse DP row by row, for o >= e: lane L holds columns c0 + L and
// c0 + 32 + L of reverse row a, where c0 is the first live column of row a - 1 (no
// cell left of it has a live predecessor).  E along the row is an exclusive prefix
// maximum over the columns to the left, taken over max(D, F): with o >= e a gap that
// E itself opened never beats extending E, and as the threshold is the same along a
// row, a gap run through a cell below it stays below it.  So the live cells and their
// values are those of the antidiagonal form.  Returns false when a row needs more
// than 64 columns.
__device__ bool band_rows(const uint8_t *__restrict__ q, const uint8_t *__restrict__ t, const int *s_mat, int o,
                          int e, int S, int ei, int ej, const int16_t *__restrict__ bm, int *amax_out,
                          int *bmax_out) {
    const int lane = threadIdx.x & 31;
    const int A = ei + 1, B = ej + 1;
    const int slack = max(o - e, 0);
    int Hp[2] = {NEG, NEG}, Fp[2] = {NEG, NEG};        // row a - 1 at columns c0p + 32 c + lane
    int c0p = 0, plo = 0, phi = -1;                     // its window start and live columns
    bool pwide = false;
    int amax = 0, bmax = 0;
    for (int a = 0; a <= A; ++a) {
        if (a > 0 && phi < plo) break;                  // row a - 1 had no live cell
        const int c0 = a == 0 ? 0 : plo;
        if (a > 0 && phi + 1 > c0 + 63) return false;   // its diagonal successors leave the window
        const int i = ei - a + 1;                       // forward row of this reverse row
        const int thr = S - (i >= 1 ? (int)bm[(i - 1) >> 1] : 0) - slack;
        const int qa = a >= 1 ? (int)q[i] * PASTIS_NSYM : 0;
        const int dsh = c0 - c0p;
        int H[2] = {NEG, NEG}, F[2] = {NEG, NEG};
        unsigned live[2] = {0u, 0u};
        int carry = NEG;                                // max of max(D, F) + k e left of the chunk
        int tb = -1;                                    // this lane's largest column reaching S
        bool wide = false;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (c == 1) {
                // the second chunk when row a - 1 reaches past the first, or an E run
                // leaves it still at or above the threshold
                const int e_next = carry - o - 31 * e;
                if (!(phi + 1 > c0 + 31 || e_next >= thr)) break;
                wide = true;
            }
            const int k = 32 * c + lane, b = c0 + k;
            const int src = k + dsh;
            const int hb = row_get(Hp, src, pwide), fb = row_get(Fp, src, pwide);
            const int hd = row_get(Hp, src - 1, pwide);
            int hh = NEG, fv = NEG;
            if (b <= B) {
                if (a >= 1) {
                    fv = max(max(hb - o, fb - e), NEG);
                    const int dv = (b >= 1 && hd != NEG) ? hd + s_mat[qa + (int)t[ej - b + 1]] : NEG;
                    hh = max(dv, fv);
                } else if (b == 0) {
                    hh = 0;                             // the end cell
                }
            }
            int incl = hh > NEG ? hh + k * e : NEG;
#pragma unroll
            for (int x = 1; x < 32; x <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, x);
                if (lane >= x) incl = max(incl, y);
            }
            int excl = __shfl_up_sync(0xffffffffu, incl, 1);
            if (lane == 0) excl = NEG;
            excl = max(excl, carry);
            carry = max(carry, __shfl_sync(0xffffffffu, incl, 31));
            const int ev = (b >= 1 && excl > NEG) ? excl - o - (k - 1) * e : NEG;
            int h = max(hh, ev);
            if (b > B || h < thr) { h = NEG; fv = NEG; }
            H[c] = h; F[c] = fv;
            live[c] = __ballot_sync(0xffffffffu, h != NEG);
            if (h == S) tb = b;
        }
        if (wide) {
            // a live run still going past the second chunk needs more than 64 columns
            if (carry - o - 63 * e >= thr) return false;
        }
        if (__any_sync(0xffffffffu, tb >= 0)) {
            amax = a;
            bmax = max(bmax, __reduce_max_sync(0xffffffffu, tb < 0 ? 0 : tb));
        }
        Hp[0] = H[0]; Hp[1] = H[1]; Fp[0] = F[0]; Fp[1] = F[1];
        c0p = c0; pwide = wide;
        if (live[0] | live[1]) {
            plo = c0 + (live[0] ? __ffs(live[0]) - 1 : 32 + __ffs(live[1]) - 1);
            phi = c0 + (live[1] ? 63 - __clz(live[1]) : 31 - __clz(live[0]));
        } else {
            plo = 1; phi = 0;
        }
    }
    *amax_out = amax;
    *bmax_out = bmax;
    return true;
}

// Pass 2 over every pair pass 1 scored: one warp per pair, a few pairs per grab.
__global__ void __launch_bounds__(SW_THREADS, 5) k_sw_bound(const uint8_t *qcodes, const int64_t *qoffsets,
                                                         const uint8_t *tcodes, const int64_t *toffsets,
                                                         const pastis_cand *pairs, int64_t n_pairs,
                                                         const int8_t *gmat, int o, int e, const int16_t *bm_all,
                                                         const int64_t *bm_off, unsigned long long *next_pair,
                                                         sw_score_out *res, int cov_cut, const int64_t *dn,
                                                         const int *chk) {
    if (dn) n_pairs = *dn;
    if (chk && (chk[0] | chk[1])) return;
    __shared__ int s_mat[PASTIS_NSYM * PASTIS_NSYM];
    for (int x = threadIdx.x; x < PASTIS_NSYM * PASTIS_NSYM; x += blockDim.x) s_mat[x] = gmat[x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    constexpr int GRAB = 8;
    for (;;) {
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(next_pair, (unsigned long long)GRAB);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= (unsigned long long)n_pairs) break;
        // lane u < GRAB fetches pair g + u's pass-1 result, sequences and bounds, so the
        // grab's load chains run side by side instead of one after the other
        int ok_l = 0, sc_l = 0, ei_l = 0, ej_l = 0;
        int64_t qo_l = 0, to_l = 0, bo_l = 0;
        const int64_t pl = (int64_t)g + lane;
        if (lane < GRAB && pl < n_pairs) {
            const sw_score_out r = res[pl];
            if (!r.big && r.score > 0) {
                const pastis_cand c = pairs[pl];
                qo_l = qoffsets[c.i];
                to_l = toffsets[c.j];
                bo_l = bm_off[pl];
                sc_l = r.score; ei_l = r.end_i; ej_l = r.end_j;
                ok_l = 1;
                // the filter-only mode: a pair whose end already rules out coverage
                if (cov_cut >= 0 &&
                    cannot_cover(r, (int)(qoffsets[c.i + 1] - qo_l), (int)(toffsets[c.j + 1] - to_l), cov_cut))
                    ok_l = 0;
            }
        }
        for (int u = 0; u < GRAB; ++u) {
            if (!__shfl_sync(0xffffffffu, ok_l, u)) continue;
            const int64_t p = (int64_t)g + u;
            const int score = __shfl_sync(0xffffffffu, sc_l, u);
            const int ei = __shfl_sync(0xffffffffu, ei_l, u), ej = __shfl_sync(0xffffffffu, ej_l, u);
            const uint8_t *qp = qcodes + __shfl_sync(0xffffffffu, qo_l, u);
            const uint8_t *tp = tcodes + __shfl_sync(0xffffffffu, to_l, u);
            const int16_t *bm = bm_all + __shfl_sync(0xffffffffu, bo_l, u);
            int amax = 0, bmax = 0;
            bool ok = o >= e && band_rows(qp, tp, s_mat, o, e, score, ei, ej, bm, &amax, &bmax);
            if (!ok) ok = band_walk(qp, tp, s_mat, o, e, score, ei, ej, bm, &amax, &bmax);
            if (ok && amax > 0 && bmax > 0 && lane == 0) {
                res[p].rect_i = ei + 1 - amax;
                res[p].rect_j = ej + 1 - bmax;
            }                                      // else: the whole up-left rectangle (0, 0)
        }
    }
}

// Row-pair bound entries of each pair: (query length + 1) / 2.
__global__ void k_bm_count(const pastis_cand *pairs, int64_t n, const int64_t *qoffsets, int64_t *cnt,
                           const int64_t *dn, const int *chk) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    // past the batch, or a batch the checks refused (its indexes are not to be followed)
    if ((dn && p >= *dn) || (chk && (chk[0] | chk[1]))) { cnt[p] = 0; return; }
    const int i = pairs[p].i;
    cnt[p] = (qoffsets[i + 1] - qoffsets[i] + 1) / 2;
}

__global__ void __launch_bounds__(SW_THREADS, 2) k_sw_score(const uint8_t *qcodes, const int64_t *qoffsets,
                                                         const uint8_t *tcodes, const int64_t *toffsets,
                                                         const pastis_cand *pairs, const int64_t *seg_start,
                                                         int64_t n_seg, const int8_t *gmat, int o, int e,
                                                         int max_s, int prow_cap, uint32_t one, char *scratch,
                                                         size_t warp_bytes, int sstride, int *next_seg,
                                                         int16_t *bm_all, const int64_t *bm_off, sw_score_out *out,
                                                         unsigned long long *cells, const uint8_t *extra,
                                                         unsigned long long *tune, const uint32_t *d_nseg,
                                                         const int *chk) {
    // captured launches: the segment count from device memory, nothing on bad input
    if (d_nseg) n_seg = *d_nseg;
    if (chk && (chk[0] | chk[1])) return;
    // dynamic shared memory: the profile [NRES][prow_cap] bytes (prow_cap a whole number of stripes)
    extern __shared__ __align__(16) uint8_t s_prof[];
    __shared__ int s_seg, s_next;
    __shared__ uint32_t s_key[SEG_MAX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * SW_WARPS + warp;
    uint2 *my = reinterpret_cast<uint2 *>(scratch + (size_t)gw * warp_bytes);
    const bool packable = o <= GAP_MAX;
    unsigned long long my_cells = 0;
    for (;;) {
        if (threadIdx.x == 0) { s_seg = atomicAdd(next_seg, 1); s_next = 0; }
        __syncthreads();
        const int64_t sg = s_seg;
        if (sg >= n_seg) break;
        const long long t_seg = tune ? clock64() : 0;
        const int64_t p0 = seg_start[sg], p1 = seg_start[sg + 1];
        const int cnt = (int)(p1 - p0);
        const int qi = pairs[p0].i;
        const int64_t qo = qoffsets[qi];
        const int m = (int)(qoffsets[qi + 1] - qo);
        const int bin = sw_bin(m);
        const bool int32_bin = extra[bin] == PASTIS_SW_INT32;    // the bin's pairs in 32-bit lanes
        const int ex = int32_bin ? 0 : extra[bin];
        int lr = rows_per_lane(m, ex);
        int prow8 = ((m + 32 * lr - 1) / (32 * lr)) * STRIPE_BYTES;     // profile bytes per residue
        if (prow8 > prow_cap && ex) {                                  // the extra stripes do not fit
            lr = rows_per_lane(m, 0);
            prow8 = ((m + 32 * lr - 1) / (32 * lr)) * STRIPE_BYTES;
        }
        // query profile: byte (st * 512 + l * 16 + r) of residue c = M[q_i][c] + o for row
        // i = st * 32 * lr + l * lr + r of the query; o - 64 for the pad residue, unused
        // slots and rows past the query
        if (prow8 <= prow_cap) {
            for (int x = threadIdx.x; x < NRES * prow8; x += blockDim.x) {
                const int c = x / prow8, rest = x - c * prow8;
                const int st = rest / STRIPE_BYTES, l = (rest % STRIPE_BYTES) / SLOT, r = rest % SLOT;
                const int i = st * 32 * lr + l * lr + r;
                s_prof[x] = (uint8_t)(int8_t)((r < lr && i < m && c < PASTIS_NSYM)
                                                  ? (int)gmat[qcodes[qo + i] * PASTIS_NSYM + c] + o : o - 64);
            }
        }
        // the segment's pairs by target length, longest first, so that the two pairs of
        // a warp match and the last pairs taken are the shortest
        if (threadIdx.x < SEG_MAX) {
            uint32_t key = 0xFFFFFFFFu;
            if ((int)threadIdx.x < cnt) {
                const int j = pairs[p0 + threadIdx.x].j;
                key = ((uint32_t)(65535 - (toffsets[j + 1] - toffsets[j])) << 7) | threadIdx.x;
            }
            s_key[threadIdx.x] = key;
        }
        __syncthreads();
        for (int k = 2; k <= SEG_MAX; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                const int x = threadIdx.x, y = x ^ jj;
                if (x < SEG_MAX && y > x) {
                    const uint32_t u = s_key[x], v = s_key[y];
                    if ((u > v) == ((x & k) == 0)) { s_key[x] = v; s_key[y] = u; }
                }
                __syncthreads();
            }
        }
        for (;;) {
            int pk = 0;
            if (lane == 0) pk = atomicAdd(&s_next, 2);
            pk = __shfl_sync(0xffffffffu, pk, 0);
            if (pk >= cnt) break;
            int64_t pp[2];
            int nn[2], st[2];                                     // st: 0 zero, 1 big, 2 run
            const uint8_t *tp[2];
            for (int u = 0; u < 2; ++u) {
                pp[u] = pk + u < cnt ? p0 + (int64_t)(s_key[pk + u] & (SEG_MAX - 1)) : -1;
                nn[u] = 0; st[u] = 0; tp[u] = tcodes;
                if (pp[u] < 0) continue;
                const pastis_cand c = pairs[pp[u]];
                const int64_t to = toffsets[c.j];
                nn[u] = (int)(toffsets[c.j + 1] - to);
                tp[u] = tcodes + to;
                if (m == 0 || nn[u] == 0) st[u] = 0;
                else if (int32_bin || !packable || prow8 > prow_cap ||
                         (int64_t)max_s * (int64_t)min(m, nn[u]) >= SCORE_MAX) st[u] = 1;
                else st[u] = 2;
            }
            end_cell res[2];
            res[0].h = res[1].h = 0;
            if (st[0] == 2 || st[1] == 2) {
                // both halves busy; a lone pair fills both
                const int ua = st[0] == 2 ? 0 : 1, ub = st[1] == 2 ? 1 : 0;
                int16_t *bma = bm_all + bm_off[pp[ua]], *bmb = bm_all + bm_off[pp[ub]];
                end_cell ea, eb;
#define PASTIS_SW_CASE(L)                                                                                       \
    case L:                                                                                                     \
        score_pair<L>(s_prof, prow8, tp[ua], nn[ua], tp[ub], nn[ub], m, o, e, one, my, sstride, bma, bmb, &ea, &eb); \
        break;
                switch (lr) {
                    PASTIS_SW_CASE(2) PASTIS_SW_CASE(3) PASTIS_SW_CASE(4) PASTIS_SW_CASE(5)
                    PASTIS_SW_CASE(6) PASTIS_SW_CASE(7) PASTIS_SW_CASE(8) PASTIS_SW_CASE(9)
                    PASTIS_SW_CASE(10) PASTIS_SW_CASE(11) PASTIS_SW_CASE(12) PASTIS_SW_CASE(13)
                    PASTIS_SW_CASE(14) PASTIS_SW_CASE(15)
                    default:
                        score_pair<16>(s_prof, prow8, tp[ua], nn[ua], tp[ub], nn[ub], m, o, e, one, my, sstride, bma,
                                       bmb, &ea, &eb);
                        break;
                }
#undef PASTIS_SW_CASE
                __syncwarp();
                if (st[ua] == 2) res[ua] = ea;
                if (st[ub] == 2 && ub != ua) res[ub] = eb;
            }
            for (int u = 0; u < 2; ++u) {
                if (pp[u] < 0) continue;
                sw_score_out r;
                r.score = 0; r.end_i = 0; r.end_j = 0; r.rect_i = 0; r.rect_j = 0; r.big = st[u] == 1;
                if (st[u] == 2) {
                    if (res[u].h > 0) { r.score = res[u].h; r.end_i = res[u].i; r.end_j = res[u].j; }
                    my_cells += (unsigned long long)m * (unsigned long long)nn[u];
                }
                if (lane == 0) out[pp[u]] = r;
            }
        }
        __syncthreads();
        if (tune && threadIdx.x == 0) atomicAdd(&tune[bin], (unsigned long long)(clock64() - t_seg));
    }
    if (lane == 0 && cells && my_cells) atomicAdd(cells, my_cells);
}

// ---------------------------------------------------------------------------------
// pass 3: carries over the rectangle (or the whole matrix for very large scores)
// ---------------------------------------------------------------------------------
constexpr int CR = 8;                  // rows per lane of the small-rectangle groups and of TRACK

struct stripe3_cell { int32_t h, f; uint32_t hb, fb, hm, fm; };

__device__ __forceinline__ uint32_t pack_rc(int r, int c) { return ((uint32_t)r << 16) | (uint32_t)c; }

// Carries begin (row << 16 | col, of the first column) and identities << 16 | matched
// columns, with CR rows per lane (a stripe is 32 * CR rows).  TRACK: also finds the
// row-major first maximum (for pairs pass 1 skipped); otherwise reports the state at
// (m-1, n-1).
template <bool TRACK, int CR>
__device__ void carry_warp(const uint8_t *__restrict__ q, int m, const uint8_t *__restrict__ t, int n,
                           const int *__restrict__ s_mat, int o, int e, stripe3_cell *scratch, int sstride,
                           int *h_out, int *ei_out, int *ej_out, uint32_t *beg_out, uint32_t *im_out) {
    const int lane = threadIdx.x & 31;
    int best = 0, brow = 0x7FFFFFFF, bcol = 0;
    uint32_t bbeg = 0, bim = 0;
    int endh = NEG;
    uint32_t endb = 0, endm = 0;
    constexpr int STRIPE = 32 * CR;
    const int nstripes = (m + STRIPE - 1) / STRIPE;
    for (int stripe = 0; stripe < nstripes; ++stripe) {
        const int row0 = stripe * STRIPE + lane * CR;
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
                              int lt, int ani, int cov, int filtered) {
    rec.score = S;
    rec.qb = (uint16_t)qb; rec.qe = (uint16_t)(ei + 1); rec.tb = (uint16_t)tb; rec.te = (uint16_t)(ej + 1);
    rec.ident = (uint16_t)ident;
    rec.cols = (uint16_t)((ei + 1 - qb) + (ej + 1 - tb) - M);
    const int span = lq <= lt ? ei + 1 - qb : ej + 1 - tb;
    const int L = lq <= lt ? lq : lt;
    rec.passes = (rec.cols > 0 && 100 * ident >= ani * (int)rec.cols && 100 * span >= cov * L) ? 1 : 0;
    if (filtered && !rec.passes) { rec.qb = rec.tb = 0; rec.ident = rec.cols = 0; }
}

__global__ void __launch_bounds__(SW_THREADS) k_sw_carry(const uint8_t *qcodes, const int64_t *qoffsets,
                                                         const uint8_t *tcodes, const int64_t *toffsets,
                                                         const pastis_cand *pairs, int64_t n_pairs,
                                                         const int8_t *gmat, int o, int e, int ani, int cov,
                                                         stripe3_cell *scratch, int sstride, int *next_pair,
                                                         const sw_score_out *res, int score_only, int filtered,
                                                         pastis_aln *out,
                                                         int *err, unsigned long long *cells,
                                                         unsigned long long *tune, const int64_t *dn,
                                                         const int *chk) {
    if (dn) n_pairs = *dn;
    if (chk && (chk[0] | chk[1])) return;
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
            if (!score_only && !g1.big && g1.score > 0 && g1.end_i + 1 - g1.rect_i <= GROWS) {
                const pastis_cand c = pairs[pg];
                const bool skip = filtered && cannot_cover(g1, (int)(qoffsets[c.i + 1] - qoffsets[c.i]),
                                                           (int)(toffsets[c.j + 1] - toffsets[c.j]), cov);
                if (!skip) {                       // a skipped pair's record comes from the loop below
                    gm = g1.end_i + 1 - g1.rect_i;
                    gn = g1.end_j + 1 - g1.rect_j;
                    gq = qcodes + qoffsets[c.i] + g1.rect_i;
                    gt = tcodes + toffsets[c.j] + g1.rect_j;
                }
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
                          (int)(gim >> 16), (int)(gim & 0xFFFF), lq, lt, ani, cov, filtered);
            out[pg] = rec;
        }
        // the others, one warp each
        for (int k = 0; k < 32 / GL; ++k) {
            const int64_t p = p0 + k;
            if (p >= n_pairs) break;
            const sw_score_out r1 = res[p];
            const pastis_cand c = pairs[p];
            const int64_t qo = qoffsets[c.i], to = toffsets[c.j];
            const int lq = (int)(qoffsets[c.i + 1] - qo), lt = (int)(toffsets[c.j + 1] - to);
            const bool skip = filtered && !r1.big && r1.score > 0 && cannot_cover(r1, lq, lt, cov);
            const bool small = !score_only && !r1.big && r1.score > 0 && r1.end_i + 1 - r1.rect_i <= GROWS;
            if (small && !skip) continue;
            pastis_aln rec;
            rec.score = 0; rec.qb = rec.qe = rec.tb = rec.te = 0; rec.ident = rec.cols = 0;
            rec.seed_used = 0; rec.passes = 0; rec.reserved = 0;
            if (r1.big) {
                const long long t_big = tune ? clock64() : 0;      // the tuner's cycles of 32-bit work
                if (lq > 0 && lt > 0) {
                    int h, bi, bj;
                    uint32_t beg, im;
                    carry_warp<true, CR>(qcodes + qo, lq, tcodes + to, lt, s_mat, o, e, my, sstride, &h, &bi, &bj, &beg,
                                         &im);
                    if (h > 0)
                        finish_record(rec, h, bi, bj, (int)(beg >> 16), (int)(beg & 0xFFFF), (int)(im >> 16),
                                      (int)(im & 0xFFFF), lq, lt, ani, cov, filtered);
                    if (score_only) { rec.qb = rec.tb = 0; rec.ident = rec.cols = 0; rec.passes = 0; }
                    if (lane == 0) my_cells += (unsigned long long)lq * lt;
                }
                if (tune && lane == 0) atomicAdd(&tune[sw_bin(lq)], (unsigned long long)(clock64() - t_big));
            } else if (r1.score > 0 && (score_only || skip)) {
                rec.score = r1.score;                       // score and end only
                rec.qe = (uint16_t)(r1.end_i + 1);
                rec.te = (uint16_t)(r1.end_j + 1);
            } else if (r1.score > 0) {
                const int ri = r1.rect_i, rj = r1.rect_j;
                int h, dummy_i, dummy_j;
                uint32_t beg, im;
                // rows per lane from the rectangle's height, so that all 32 lanes have rows
                const int rows = r1.end_i + 1 - ri;
                const int ns3 = (rows + 32 * CR - 1) / (32 * CR);
                const int cr = min(CR, max(2, (((rows + 32 * ns3 - 1) / (32 * ns3)) + 1) & ~1));
                const uint8_t *cq = qcodes + qo + ri, *ct = tcodes + to + rj;
                const int cn = r1.end_j + 1 - rj;
#define PASTIS_CARRY_CASE(C) \
    case C: carry_warp<false, C>(cq, rows, ct, cn, s_mat, o, e, my, sstride, &h, &dummy_i, &dummy_j, &beg, &im); break;
                switch (cr) {
                    PASTIS_CARRY_CASE(2) PASTIS_CARRY_CASE(4) PASTIS_CARRY_CASE(6)
                    default: carry_warp<false, CR>(cq, rows, ct, cn, s_mat, o, e, my, sstride, &h, &dummy_i, &dummy_j,
                                                   &beg, &im); break;
                }
#undef PASTIS_CARRY_CASE
                if (h != r1.score && lane == 0) atomicExch(err, 1);
                finish_record(rec, r1.score, r1.end_i, r1.end_j, ri + (int)(beg >> 16), rj + (int)(beg & 0xFFFF),
                              (int)(im >> 16), (int)(im & 0xFFFF), lq, lt, ani, cov, filtered);
            }
            if (lane == 0) out[p] = rec;
        }
    }
    if (lane == 0 && cells && my_cells) atomicAdd(cells, my_cells);
}

}  // namespace

cudaError_t sw_set_smem_limit(size_t bytes) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_sw_score);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_sw_score, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(bytes - fa.sharedSizeBytes));
}

// Host side of the Smith-Waterman path (called by pastis_align_pairs after validation).
// dn != nullptr: a captured launch sequence (no host synchronisation): n_pairs is the
// capacity, the pair count is *dn in device memory, the row-pair bounds take their
// capacity bound, and chk (the input checks' flags) stops the kernels on bad input.
pastis_status sw_align(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets, const uint8_t *d_tcodes,
                       const int64_t *d_toffsets, const pastis_cand *d_pairs,
                       int64_t n_pairs, const pastis_params *p, const int8_t *dmat, int *flags, int lmax,
                       pastis_aln *d_out, int64_t *d_cells, const int64_t *dn, const int *chk) {
    cudaStream_t st = ctx->stream;
    int max_s = 0;
    for (int x = 0; x < PASTIS_NSYM * PASTIS_NSYM; ++x) max_s = std::max(max_s, (int)p->matrix[x]);
    // segments of pairs sharing a query
    uint32_t *sflags;
    PASTIS_WS(sflags, ctx, WS_ALN_ORDER, sizeof(uint32_t) * (2 * (size_t)n_pairs + 2) + sizeof(int64_t) * (n_pairs + 2) + 16);
    uint32_t *soff = sflags + n_pairs + 1;
    int64_t *seg_start = (int64_t *)(((uintptr_t)(soff + n_pairs + 1) + 7) & ~(uintptr_t)7);
    k_seg_flags<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(d_pairs, n_pairs, sflags, dn);
    PASTIS_LAUNCHED(ctx);
    pastis_status s = exclusive_scan_u32(ctx, sflags, soff, n_pairs);
    if (s != PASTIS_OK) return s;
    k_seg_starts<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(sflags, soff, n_pairs, seg_start, dn);
    PASTIS_LAUNCHED(ctx);
    uint32_t h_nseg = 0;
    if (!dn) {
        PASTIS_CUDA_TRY(cudaMemcpyAsync(&h_nseg, soff + n_pairs, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    }

    // row-pair bounds of pass 1 for pass 2: (query length + 1) / 2 int16 per pair
    int64_t *bm_cnt;
    PASTIS_WS(bm_cnt, ctx, WS_ALN_BOFF, sizeof(int64_t) * (2 * (size_t)n_pairs + 1));
    int64_t *bm_off = bm_cnt + n_pairs;
    k_bm_count<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(d_pairs, n_pairs, d_qoffsets, bm_cnt, dn, chk);
    PASTIS_LAUNCHED(ctx);
    s = exclusive_scan_i64(ctx, bm_cnt, bm_off, n_pairs);
    if (s != PASTIS_OK) return s;
    int64_t h_bm = n_pairs * (int64_t)((lmax + 1) / 2);     // the bound of a captured sequence
    if (!dn) {
        PASTIS_CUDA_TRY(cudaMemcpyAsync(&h_bm, bm_off + n_pairs, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    int16_t *bm_all;
    PASTIS_WS(bm_all, ctx, WS_ALN_BOUND, sizeof(int16_t) * (size_t)h_bm + 16);

    sw_score_out *res;
    PASTIS_WS(res, ctx, WS_ALN_PASS1, sizeof(sw_score_out) * (size_t)n_pairs);
    // pass 1+2: profile rows up to the longest query (in whole stripes), within shared memory
    int max_extra = 0;
    for (int b = 0; b < PASTIS_SW_BINS; ++b) max_extra = std::max(max_extra, (int)ctx->sw_lay.extra[b]);
    int prow_cap = ((lmax + STRIPE1 - 1) / STRIPE1 + max_extra) * STRIPE1;
    if (prow_cap < STRIPE1) prow_cap = STRIPE1;
    auto shm_for = [](int pc) { return (size_t)NRES * pc; };
    while (prow_cap > STRIPE1 && shm_for(prow_cap) + 1024 > ctx->smem_optin) prow_cap -= STRIPE1;
    const size_t shm1 = shm_for(prow_cap);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sw_score, SW_THREADS, shm1);
    if (per_sm < 1) per_sm = 1;
    const int blocks1 = ctx->sm_count * per_sm;
    const int sstride = lmax + 1;
    const size_t warp_bytes = (sizeof(uint2) * 2 * (size_t)sstride + 255) & ~(size_t)255;
    const size_t scr1 = warp_bytes * (size_t)blocks1 * SW_WARPS;
    const int blocks3 = ctx->sm_count * 2;
    const size_t scr3 = sizeof(stripe3_cell) * (size_t)blocks3 * SW_WARPS * 2 * sstride;
    void *scratch;
    PASTIS_WS(scratch, ctx, WS_ALN_SCRATCH, std::max(scr1, scr3));
    prof_begin(ctx, "sw_pass1");
    k_sw_score<<<blocks1, SW_THREADS, shm1, st>>>(d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs, seg_start,
                                                  (int64_t)h_nseg, dmat,
                                                  p->gap_open, p->gap_extend, max_s, prow_cap, 1u, (char *)scratch,
                                                  warp_bytes, sstride, flags + 1, bm_all, bm_off, res,
                                                  (unsigned long long *)d_cells, (const uint8_t *)dmat + 640,
                                                  ctx->d_tune, dn ? soff + n_pairs : nullptr, chk);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    const int score_only = p->mode == PASTIS_SW_SCORE;
    const int filtered = p->mode == PASTIS_SW_FILTERED;
    int per_sm2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_sw_bound, SW_THREADS, 0);
    if (per_sm2 < 1) per_sm2 = 1;
    if (!score_only) {                         // the score mode needs no begin, so no rectangle
        prof_begin(ctx, "sw_pass2");
        k_sw_bound<<<ctx->sm_count * per_sm2, SW_THREADS, 0, st>>>(d_qcodes, d_qoffsets, d_tcodes, d_toffsets,
                                                                   d_pairs, n_pairs, dmat, p->gap_open, p->gap_extend,
                                                                   bm_all, bm_off, (unsigned long long *)(flags + 10),
                                                                   res, filtered ? p->cov_min_pct : -1, dn, chk);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    prof_begin(ctx, "sw_pass3");
    k_sw_carry<<<blocks3, SW_THREADS, 0, st>>>(d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs, n_pairs, dmat,
                                               p->gap_open,
                                               p->gap_extend, p->ani_min_pct, p->cov_min_pct,
                                               (stripe3_cell *)scratch, sstride, flags + 8, res, score_only, filtered,
                                               d_out, flags,
                                               (unsigned long long *)d_cells, ctx->d_tune, dn, chk);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    return PASTIS_OK;
}
