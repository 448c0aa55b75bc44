// a8-a9: Smith-Waterman and x-drop alignment of candidate pairs (Sec. IV-E, Sec. VI).
//
// Smith-Waterman, affine gaps (a gap of length L costs open + (L-1)*extend):
//   E(i,j) = max(H(i,j-1) - o, E(i,j-1) - e)     F(i,j) = max(H(i-1,j) - o, F(i-1,j) - e)
//   H(i,j) = max(0, H(i-1,j-1) + s(q_i, t_j), F(i,j), E(i,j))
// The reported alignment is the one a traceback from the end cell (the first maximum
// in row-major order) selects when it prefers the diagonal, then F, then E, and a gap
// open over an extension.  The GPU never traces back: every state carries, along the
// predecessor that traceback would take, the statistic it needs, so the value held at
// the end cell is the traceback's.
//
// Two passes over a warp wavefront:
//   pass 1 (whole matrix) carries the alignment's begin cell; it gives score, end and
//          begin, hence both spans, for every pair;
//   pass 2 (only the rectangle [qb, qe) x [tb, te)) carries identities and matched
//          columns.  Inside that rectangle, with zero boundaries, every cell of the
//          traced path keeps its value and every choice along it stays the same, so
//          the carried statistic at the end cell is the full matrix's.  Random pairs
//          have short alignments, so pass 2 costs little.
// Wavefront: lane l of a warp owns R consecutive query rows; at step s it computes
// column j = s - l for its rows, taking the bottom H/F (and carries) of lane l-1's
// previous step through __shfl_up_sync.  Queries longer than 32R rows are done in
// stripes; the last row of a stripe goes to the next through a per-warp buffer.
//
// x-drop (XD): from a seed, the seed's score plus two anchored extensions (right of
// the seed, and left of it on the reversed prefixes), each computed antidiagonal by
// antidiagonal by one warp: cells of antidiagonal d+1 are those adjacent to the live
// range of d, a cell dies when H < best - X (best over the earlier antidiagonals),
// and the extension ends when an antidiagonal has no live cell.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int NEG = -1000000000;
constexpr int ALN_THREADS = 256;
constexpr int ALN_WARPS = ALN_THREADS / 32;
constexpr int SW_R = 8;                  // query rows per lane
constexpr int STRIPE = 32 * SW_R;
constexpr int PAD_CODE = PASTIS_NSYM;    // score row for rows past the end of the query
constexpr int PAD_SCORE = -30000;

struct sw_pass1_out {                     // per pair
    int32_t score;
    uint32_t end;                         // (row << 16) | col
    uint32_t begin;                       // (row << 16) | col
    int32_t pad;
};

__device__ __forceinline__ uint32_t pack_rc(int r, int c) { return ((uint32_t)r << 16) | (uint32_t)c; }

// Scratch row handed between stripes: H, F and their carries for every column.
struct stripe_cell { int32_t h, f; uint32_t hc, fc; };

// One warp computes one matrix.  MODE 1: carry = begin cell; tracks the first maximum.
// MODE 2: carry = ident << 16 | matched columns; reports the carry at (m-1, n-1).
template <int MODE>
__device__ void sw_warp(const uint8_t *__restrict__ q, int m, const uint8_t *__restrict__ t, int n,
                        const int *__restrict__ s_mat, int o, int e, stripe_cell *scratch, int sstride,
                        int *best_out,
                        int *best_row_out, int *best_col_out, uint32_t *best_carry_out) {
    const int lane = threadIdx.x & 31;
    int best = 0, best_row = 0x7FFFFFFF, best_col = 0;
    uint32_t best_carry = 0;
    int end_h = NEG;
    uint32_t end_c = 0;
    const int nstripes = (m + STRIPE - 1) / STRIPE;
    for (int stripe = 0; stripe < nstripes; ++stripe) {
        const int row0 = stripe * STRIPE + lane * SW_R;
        int qoff[SW_R];
        int Hc[SW_R], Ec[SW_R];
        uint32_t HCc[SW_R], ECc[SW_R];
#pragma unroll
        for (int r = 0; r < SW_R; ++r) {
            const int i = row0 + r;
            qoff[r] = (i < m ? (int)q[i] : PAD_CODE) * 32;
            Hc[r] = 0;
            Ec[r] = NEG;
            HCc[r] = MODE == 1 ? pack_rc(i + 1, 0) : 0u;
            ECc[r] = 0;
        }
        int dtop_h = 0;                                   // H(row0-1, j-1)
        uint32_t dtop_c = MODE == 1 ? pack_rc(row0, 0) : 0u;
        int out_h = 0, out_f = NEG, out_t = 0;
        uint32_t out_hc = 0, out_fc = 0;
        const stripe_cell *in_buf = scratch + (size_t)(stripe & 1) * sstride;
        stripe_cell *out_buf = scratch + (size_t)((stripe + 1) & 1) * sstride;
        const bool last_stripe = stripe + 1 == nstripes;
        const int nsteps = n + 31;
        for (int s = 0; s < nsteps; ++s) {
            const int j = s - lane;
            int up_h = __shfl_up_sync(0xffffffffu, out_h, 1);
            int up_f = __shfl_up_sync(0xffffffffu, out_f, 1);
            uint32_t up_hc = __shfl_up_sync(0xffffffffu, out_hc, 1);
            uint32_t up_fc = __shfl_up_sync(0xffffffffu, out_fc, 1);
            int tj = __shfl_up_sync(0xffffffffu, out_t, 1);
            if (lane == 0 && j < n) {
                tj = t[j];
                if (stripe == 0) {
                    up_h = 0; up_f = NEG;
                    up_hc = MODE == 1 ? pack_rc(0, j + 1) : 0u;
                    up_fc = 0;
                } else {
                    stripe_cell c = in_buf[j];
                    up_h = c.h; up_f = c.f; up_hc = c.hc; up_fc = c.fc;
                }
            }
            if (j >= 0 && j < n) {
                int dh = dtop_h;
                uint32_t dc = dtop_c;
                int ah = up_h;
                uint32_t ac = up_hc;
                int f = up_f;
                uint32_t fc = up_fc;
#pragma unroll
                for (int r = 0; r < SW_R; ++r) {
                    const int i = row0 + r;
                    // E: horizontal gap, from (i, j-1)
                    const int eo = Hc[r] - o, ex = Ec[r] - e;
                    const bool eopen = eo >= ex;
                    const int ev = eopen ? eo : ex;
                    const uint32_t evc = eopen ? HCc[r] : ECc[r];
                    // F: vertical gap, from (i-1, j)
                    const int fo = ah - o, fx = f - e;
                    const bool fopen = fo >= fx;
                    f = fopen ? fo : fx;
                    fc = fopen ? ac : fc;
                    // H: diagonal > F > E, restart at 0
                    const int sc = s_mat[qoff[r] + tj];
                    int h = dh + sc;
                    uint32_t hc;
                    if (MODE == 1) hc = dc;
                    else hc = dc + ((qoff[r] == tj * 32) ? 0x10001u : 1u);
                    if (f > h) { h = f; hc = fc; }
                    if (ev > h) { h = ev; hc = evc; }
                    if (h <= 0) { h = 0; hc = MODE == 1 ? pack_rc(i + 1, j + 1) : 0u; }
                    if (MODE == 1) {
                        if (i < m && (h > best || (h == best && h > 0 && i < best_row))) {
                            best = h; best_row = i; best_col = j; best_carry = hc;
                        }
                    } else {
                        if (i == m - 1 && j == n - 1) { end_h = h; end_c = hc; }
                    }
                    dh = Hc[r];
                    dc = HCc[r];
                    Hc[r] = h; HCc[r] = hc;
                    Ec[r] = ev; ECc[r] = evc;
                    ah = h; ac = hc;
                }
                dtop_h = up_h;
                dtop_c = up_hc;
                out_h = ah; out_hc = ac; out_f = f; out_fc = fc; out_t = tj;
                if (lane == 31 && !last_stripe) out_buf[j] = stripe_cell{ah, f, ac, fc};
            }
        }
        __syncwarp();
    }
    if (MODE == 1) {
        // first maximum in row-major order across the warp
        for (int d = 16; d > 0; d >>= 1) {
            int ob = __shfl_xor_sync(0xffffffffu, best, d);
            int orow = __shfl_xor_sync(0xffffffffu, best_row, d);
            int ocol = __shfl_xor_sync(0xffffffffu, best_col, d);
            uint32_t oc = __shfl_xor_sync(0xffffffffu, best_carry, d);
            bool take = ob > best || (ob == best && (orow < best_row || (orow == best_row && ocol < best_col)));
            if (take) { best = ob; best_row = orow; best_col = ocol; best_carry = oc; }
        }
        *best_out = best; *best_row_out = best_row; *best_col_out = best_col; *best_carry_out = best_carry;
    } else {
        for (int d = 16; d > 0; d >>= 1) {
            int oh = __shfl_xor_sync(0xffffffffu, end_h, d);
            uint32_t oc = __shfl_xor_sync(0xffffffffu, end_c, d);
            if (oh > end_h) { end_h = oh; end_c = oc; }
        }
        *best_out = end_h; *best_carry_out = end_c;
    }
}

__device__ void load_matrix(const int8_t *gmat, int *s_mat) {
    for (int x = threadIdx.x; x < (PASTIS_NSYM + 1) * 32; x += blockDim.x) {
        int a = x / 32, b = x % 32;
        s_mat[x] = (a < PASTIS_NSYM && b < PASTIS_NSYM) ? (int)gmat[a * PASTIS_NSYM + b] : PAD_SCORE;
    }
}

__global__ void __launch_bounds__(ALN_THREADS) k_sw_pass1(const uint8_t *codes, const int64_t *offsets,
                                                          const pastis_cand *pairs, int64_t n_pairs,
                                                          const int8_t *gmat, int o, int e,
                                                          stripe_cell *scratch, int sstride, int *next_pair,
                                                          sw_pass1_out *out, unsigned long long *cells) {
    __shared__ int s_mat[(PASTIS_NSYM + 1) * 32];
    load_matrix(gmat, s_mat);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * ALN_WARPS + (threadIdx.x >> 5);
    stripe_cell *my = scratch + (size_t)gw * 2 * sstride;
    unsigned long long my_cells = 0;
    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(next_pair, 1);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= n_pairs) break;
        const pastis_cand c = pairs[p];
        const int64_t qo = offsets[c.i], to = offsets[c.j];
        const int m = (int)(offsets[c.i + 1] - qo), n = (int)(offsets[c.j + 1] - to);
        int best = 0, brow = 0, bcol = 0;
        uint32_t bc = 0;
        if (m > 0 && n > 0)
            sw_warp<1>(codes + qo, m, codes + to, n, s_mat, o, e, my, sstride, &best, &brow, &bcol, &bc);
        if (lane == 0) {
            sw_pass1_out r;
            r.score = best;
            r.end = best > 0 ? pack_rc(brow, bcol) : 0u;
            r.begin = best > 0 ? bc : 0u;
            r.pad = 0;
            out[p] = r;
            my_cells += (unsigned long long)m * (unsigned long long)n;
        }
    }
    if (lane == 0 && cells) atomicAdd(cells, my_cells);
}

__global__ void __launch_bounds__(ALN_THREADS) k_sw_pass2(const uint8_t *codes, const int64_t *offsets,
                                                          const pastis_cand *pairs, int64_t n_pairs,
                                                          const int8_t *gmat, int o, int e, int ani, int cov,
                                                          stripe_cell *scratch, int sstride, int *next_pair,
                                                          const sw_pass1_out *p1, pastis_aln *out, int *err) {
    __shared__ int s_mat[(PASTIS_NSYM + 1) * 32];
    load_matrix(gmat, s_mat);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * ALN_WARPS + (threadIdx.x >> 5);
    stripe_cell *my = scratch + (size_t)gw * 2 * sstride;
    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(next_pair, 1);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= n_pairs) break;
        const pastis_cand c = pairs[p];
        const sw_pass1_out r1 = p1[p];
        pastis_aln rec;
        rec.score = 0; rec.qb = rec.qe = rec.tb = rec.te = 0; rec.ident = rec.cols = 0;
        rec.seed_used = 0; rec.passes = 0; rec.reserved = 0;
        if (r1.score > 0) {
            const int64_t qo = offsets[c.i], to = offsets[c.j];
            const int lq = (int)(offsets[c.i + 1] - qo), lt = (int)(offsets[c.j + 1] - to);
            const int qb = (int)(r1.begin >> 16), tb = (int)(r1.begin & 0xFFFF);
            const int qe = (int)(r1.end >> 16) + 1, te = (int)(r1.end & 0xFFFF) + 1;
            int endh = 0, dummy_r = 0, dummy_c = 0;
            uint32_t carry = 0;
            sw_warp<2>(codes + qo + qb, qe - qb, codes + to + tb, te - tb, s_mat, o, e, my, sstride, &endh, &dummy_r,
                       &dummy_c, &carry);
            const int M = (int)(carry & 0xFFFF), ident = (int)(carry >> 16);
            rec.score = r1.score;
            rec.qb = (uint16_t)qb; rec.qe = (uint16_t)qe; rec.tb = (uint16_t)tb; rec.te = (uint16_t)te;
            rec.ident = (uint16_t)ident;
            rec.cols = (uint16_t)((qe - qb) + (te - tb) - M);
            if (endh != r1.score && lane == 0) atomicExch(err, 1);
            const int span = lq <= lt ? qe - qb : te - tb;
            const int L = lq <= lt ? lq : lt;
            rec.passes = (rec.cols > 0 && 100 * (int)rec.ident >= ani * (int)rec.cols && 100 * span >= cov * L) ? 1 : 0;
        }
        if (lane == 0) out[p] = rec;
    }
}

// ---------------------------------------------------------------------------------
// x-drop extension
// ---------------------------------------------------------------------------------
struct ext_out {
    int32_t score;
    int32_t a, b;
    uint32_t carry;       // ident << 16 | matched columns
    int64_t cells;
};

struct xd_bufs {          // per warp, three rotating antidiagonals of (A+2) cells
    int32_t *H, *E, *F;
    uint32_t *HC, *EC, *FC;
};

// qs/ts = +1 for the right extension, -1 for the left one (q[0] is the first residue).
__device__ void xd_extend_warp(const uint8_t *q, int A, int qs, const uint8_t *t, int B, int ts,
                               const int *s_mat, int o, int e, int X, xd_bufs buf, int W, ext_out *res) {
    const int lane = threadIdx.x & 31;
    int lo[3], hi[3];                       // computed range of the three antidiagonals
    // antidiagonal 0: the anchor
    if (lane == 0) {
        buf.H[0] = 0; buf.E[0] = NEG; buf.F[0] = NEG;
        buf.HC[0] = 0; buf.EC[0] = 0; buf.FC[0] = 0;
    }
    __syncwarp();
    lo[0] = 0; hi[0] = 0;
    lo[1] = 1; hi[1] = 0;                   // empty
    lo[2] = 1; hi[2] = 0;
    int best = 0, ba = 0, bb = 0;
    uint32_t bc = 0;
    long long cells = 1;
    int llo = 0, lhi = 0;
    for (int d = 1; d <= A + B; ++d) {
        int clo = max(max(llo, d - B), 0);
        int chi = min(min(lhi + 1, A), d);
        if (clo > chi) break;
        const int sc = d % 3, s1 = (d + 2) % 3, s2 = (d + 1) % 3;   // sets of d, d-1, d-2
        int32_t *Hd = buf.H + sc * W, *Ed = buf.E + sc * W, *Fd = buf.F + sc * W;
        uint32_t *HCd = buf.HC + sc * W, *ECd = buf.EC + sc * W, *FCd = buf.FC + sc * W;
        const int32_t *H1 = buf.H + s1 * W, *E1 = buf.E + s1 * W, *F1 = buf.F + s1 * W;
        const uint32_t *HC1 = buf.HC + s1 * W, *EC1 = buf.EC + s1 * W, *FC1 = buf.FC + s1 * W;
        const int32_t *H2 = buf.H + s2 * W;
        const uint32_t *HC2 = buf.HC + s2 * W;
        const int lo1 = lo[s1], hi1 = hi[s1], lo2 = lo[s2], hi2 = hi[s2];
        int my_lo = 0x7FFFFFFF, my_hi = -1, my_best = NEG, my_ba = 0;
        uint32_t my_bc = 0;
        for (int a = clo + lane; a <= chi; a += 32) {
            const int b = d - a;
            int ev = NEG, fv = NEG, dv = NEG;
            uint32_t evc = 0, fvc = 0, dvc = 0;
            if (b >= 1 && a >= lo1 && a <= hi1) {
                const int eo = H1[a] - o, ex = E1[a] - e;
                if (eo >= ex) { ev = eo; evc = HC1[a]; } else { ev = ex; evc = EC1[a]; }
                if (ev < NEG) ev = NEG;
            }
            if (a >= 1 && a - 1 >= lo1 && a - 1 <= hi1) {
                const int fo = H1[a - 1] - o, fx = F1[a - 1] - e;
                if (fo >= fx) { fv = fo; fvc = HC1[a - 1]; } else { fv = fx; fvc = FC1[a - 1]; }
                if (fv < NEG) fv = NEG;
            }
            if (a >= 1 && b >= 1 && a - 1 >= lo2 && a - 1 <= hi2) {
                const int hd = H2[a - 1];
                if (hd != NEG) {
                    const int qa = q[(long long)(a - 1) * qs], tb = t[(long long)(b - 1) * ts];
                    dv = hd + s_mat[qa * 32 + tb];
                    dvc = HC2[a - 1] + (qa == tb ? 0x10001u : 1u);
                }
            }
            int h = dv;
            uint32_t hc = dvc;
            if (fv > h) { h = fv; hc = fvc; }
            if (ev > h) { h = ev; hc = evc; }
            if (h < best - X) { h = NEG; ev = NEG; fv = NEG; }
            Hd[a] = h; Ed[a] = ev; Fd[a] = fv;
            HCd[a] = hc; ECd[a] = evc; FCd[a] = fvc;
            if (h != NEG) {
                my_lo = min(my_lo, a);
                my_hi = max(my_hi, a);
                if (h > my_best) { my_best = h; my_ba = a; my_bc = hc; }
            }
        }
        cells += chi - clo + 1;
        lo[sc] = clo; hi[sc] = chi;
        for (int x = 16; x > 0; x >>= 1) {
            my_lo = min(my_lo, __shfl_xor_sync(0xffffffffu, my_lo, x));
            my_hi = max(my_hi, __shfl_xor_sync(0xffffffffu, my_hi, x));
            const int ob = __shfl_xor_sync(0xffffffffu, my_best, x);
            const int oa = __shfl_xor_sync(0xffffffffu, my_ba, x);
            const uint32_t oc = __shfl_xor_sync(0xffffffffu, my_bc, x);
            if (ob > my_best || (ob == my_best && oa < my_ba)) { my_best = ob; my_ba = oa; my_bc = oc; }
        }
        __syncwarp();
        if (my_hi < 0) break;
        if (my_best > best) { best = my_best; ba = my_ba; bb = d - my_ba; bc = my_bc; }
        llo = my_lo; lhi = my_hi;
    }
    res->score = best; res->a = ba; res->b = bb; res->carry = bc; res->cells = cells;
}

__global__ void __launch_bounds__(ALN_THREADS) k_xd_ext(const uint8_t *codes, const int64_t *offsets,
                                                        const pastis_cand *pairs, int64_t n_pairs, int k,
                                                        const int8_t *gmat, int o, int e, int X, int32_t *gbuf,
                                                        int W, int *next_task, ext_out *out) {
    __shared__ int s_mat[(PASTIS_NSYM + 1) * 32];
    load_matrix(gmat, s_mat);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * ALN_WARPS + (threadIdx.x >> 5);
    xd_bufs buf;
    int32_t *base = gbuf + (size_t)gw * 18 * W;
    buf.H = base; buf.E = base + 3 * W; buf.F = base + 6 * W;
    buf.HC = (uint32_t *)(base + 9 * W); buf.EC = (uint32_t *)(base + 12 * W); buf.FC = (uint32_t *)(base + 15 * W);
    const int64_t ntask = n_pairs * 4;
    for (;;) {
        int64_t task = 0;
        if (lane == 0) task = atomicAdd((unsigned long long *)next_task, 1ull);
        task = __shfl_sync(0xffffffffu, task, 0);
        if (task >= ntask) break;
        const int64_t p = task >> 2;
        const int seed = (int)((task >> 1) & 1), left = (int)(task & 1);
        const pastis_cand c = pairs[p];
        ext_out r;
        r.score = 0; r.a = 0; r.b = 0; r.carry = 0; r.cells = 0;
        const bool has = seed == 0 || (c.count >= 2 && c.qpos[1] != 0xFFFF);
        if (has) {
            const int64_t qo = offsets[c.i], to = offsets[c.j];
            const int lq = (int)(offsets[c.i + 1] - qo), lt = (int)(offsets[c.j + 1] - to);
            const int pi = c.qpos[seed], pj = c.tpos[seed];
            if (!left)
                xd_extend_warp(codes + qo + pi + k, lq - pi - k, 1, codes + to + pj + k, lt - pj - k, 1, s_mat, o,
                               e, X, buf, W, &r);
            else
                xd_extend_warp(codes + qo + pi - 1, pi, -1, codes + to + pj - 1, pj, -1, s_mat, o, e, X, buf, W,
                               &r);
        }
        if (lane == 0) out[task] = r;
        __syncwarp();
    }
}

__global__ void k_xd_combine(const uint8_t *codes, const int64_t *offsets, const pastis_cand *pairs,
                             int64_t n_pairs, int k, const int8_t *gmat, int ani, int cov, const ext_out *ext,
                             pastis_aln *out, unsigned long long *cells) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long my = 0;
    if (p < n_pairs) {
        const pastis_cand c = pairs[p];
        const int64_t qo = offsets[c.i], to = offsets[c.j];
        const int lq = (int)(offsets[c.i + 1] - qo), lt = (int)(offsets[c.j + 1] - to);
        const int ns = (c.count >= 2 && c.qpos[1] != 0xFFFF) ? 2 : 1;
        pastis_aln best;
        bool best_ok = false;
        for (int s = 0; s < ns; ++s) {
            const ext_out R = ext[p * 4 + s * 2 + 0], L = ext[p * 4 + s * 2 + 1];
            const int pi = c.qpos[s], pj = c.tpos[s];
            int seed = 0, sid = 0;
            for (int x = 0; x < k; ++x) {
                const int a = codes[qo + pi + x], b = codes[to + pj + x];
                seed += gmat[a * PASTIS_NSYM + b];
                sid += (a == b);
            }
            pastis_aln cur;
            cur.score = L.score + seed + R.score;
            cur.qb = (uint16_t)(pi - L.a); cur.tb = (uint16_t)(pj - L.b);
            cur.qe = (uint16_t)(pi + k + R.a); cur.te = (uint16_t)(pj + k + R.b);
            const int M = (int)(L.carry & 0xFFFF) + k + (int)(R.carry & 0xFFFF);
            const int ident = (int)(L.carry >> 16) + sid + (int)(R.carry >> 16);
            const int span_q = cur.qe - cur.qb, span_t = cur.te - cur.tb;
            cur.ident = (uint16_t)ident;
            cur.cols = (uint16_t)(span_q + span_t - M);
            const int span = lq <= lt ? span_q : span_t;
            const int Ls = lq <= lt ? lq : lt;
            const bool ok = cur.cols > 0 && 100 * ident >= ani * (int)cur.cols && 100 * span >= cov * Ls;
            cur.seed_used = (uint8_t)s; cur.passes = ok ? 1 : 0; cur.reserved = 0;
            bool take;
            if (s == 0) take = true;
            else if (ok != best_ok) take = ok;
            else take = cur.score > best.score;
            if (take) { best = cur; best_ok = ok; }
            my += (unsigned long long)(L.cells + R.cells);
        }
        out[p] = best;
    }
    if (cells) {
        for (int x = 16; x > 0; x >>= 1) my += __shfl_xor_sync(0xffffffffu, my, x);
        if ((threadIdx.x & 31) == 0 && my) atomicAdd(cells, my);
    }
}

__global__ void k_max_len(const int64_t *offsets, int32_t n, int *mx) {
    int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    int v = 0;
    if (s < n) v = (int)(offsets[s + 1] - offsets[s]);
    for (int x = 16; x > 0; x >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, x));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, v);
}

__global__ void k_check_codes(const uint8_t *codes, int64_t n, int *bad) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        if (codes[x] >= PASTIS_NSYM) *bad = 1;
}

__global__ void k_check_pairs(const pastis_cand *pairs, int64_t n_pairs, const int64_t *offsets, int32_t n_seq,
                              int k, int xd, int *bad) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const pastis_cand c = pairs[p];
    if (c.i < 0 || c.j < 0 || c.i >= n_seq || c.j >= n_seq) { *bad = 1; return; }
    if (!xd) return;
    const int lq = (int)(offsets[c.i + 1] - offsets[c.i]), lt = (int)(offsets[c.j + 1] - offsets[c.j]);
    const int ns = (c.count >= 2 && c.qpos[1] != 0xFFFF) ? 2 : 1;
    for (int s = 0; s < ns; ++s)
        if ((int)c.qpos[s] + k > lq || (int)c.tpos[s] + k > lt) *bad = 1;
}

}  // namespace

extern "C" pastis_status pastis_align_pairs(pastis_ctx *ctx, const uint8_t *d_codes, const int64_t *d_offsets,
                                            int32_t n_seqs, const pastis_cand *d_pairs, int64_t n_pairs,
                                            const pastis_params *params, pastis_aln *d_out, int64_t *d_cells) {
    if (!ctx || n_pairs < 0 || n_seqs < 0) return PASTIS_ERR_INVALID_ARG;
    pastis_status s = check_params(params);
    if (s != PASTIS_OK) return s;
    if (n_pairs == 0) return PASTIS_OK;
    if (!d_codes || !d_offsets || !d_pairs || !d_out || n_seqs == 0) return PASTIS_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    int8_t *dmat;
    PASTIS_WS(dmat, ctx, WS_FLAGS, 1024);
    int *flags = (int *)(dmat + 768);   // [0] error, [1] [3] pair counters, [2] max length, [4] bad pair,
                                        // [5] bad code, [6..7] task counter
    PASTIS_CUDA_TRY(cudaMemcpyAsync(dmat, params->matrix, 576, cudaMemcpyHostToDevice, st));
    PASTIS_CUDA_TRY(cudaMemsetAsync(flags, 0, 64, st));
    const int xd = params->mode == PASTIS_XD;
    k_max_len<<<(unsigned)ceil_div64(n_seqs, 256), 256, 0, st>>>(d_offsets, n_seqs, flags + 2);
    PASTIS_LAUNCHED(ctx);
    k_check_pairs<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(d_pairs, n_pairs, d_offsets, n_seqs,
                                                                     params->k, xd, flags + 4);
    PASTIS_LAUNCHED(ctx);
    int64_t h_off_end = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&h_off_end, d_offsets + n_seqs, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_off_end > 0) {
        int blocks_c = (int)std::min<int64_t>(ceil_div64(h_off_end, 256), (int64_t)ctx->sm_count * 16);
        prof_begin(ctx, "align_checks");
        k_check_codes<<<blocks_c, 256, 0, st>>>(d_codes, h_off_end, flags + 5);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    int hf[6];
    PASTIS_CUDA_TRY(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hf[4]) return PASTIS_ERR_INVALID_ARG;
    if (hf[5]) return PASTIS_ERR_INVALID_RESIDUE;
    const int lmax = hf[2];
    if (lmax > PASTIS_MAX_LEN) return PASTIS_ERR_INVALID_ARG;
    const int blocks = ctx->sm_count * 2;
    const int nwarps = blocks * ALN_WARPS;
    if (!xd) {
        const int sstride = lmax + 1;
        stripe_cell *scratch;
        PASTIS_WS(scratch, ctx, WS_ALN_SCRATCH, sizeof(stripe_cell) * (size_t)nwarps * 2 * sstride);
        sw_pass1_out *p1;
        PASTIS_WS(p1, ctx, WS_ALN_PASS1, sizeof(sw_pass1_out) * (size_t)n_pairs);
        prof_begin(ctx, "sw_pass1");
        k_sw_pass1<<<blocks, ALN_THREADS, 0, st>>>(d_codes, d_offsets, d_pairs, n_pairs, dmat, params->gap_open,
                                                   params->gap_extend, scratch, sstride, flags + 1, p1,
                                                   (unsigned long long *)d_cells);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
        prof_begin(ctx, "sw_pass2");
        k_sw_pass2<<<blocks, ALN_THREADS, 0, st>>>(d_codes, d_offsets, d_pairs, n_pairs, dmat, params->gap_open,
                                                   params->gap_extend, params->ani_min_pct, params->cov_min_pct,
                                                   scratch, sstride, flags + 3, p1, d_out, flags);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    } else {
        const int W = lmax + 2;
        int32_t *gbuf;
        PASTIS_WS(gbuf, ctx, WS_ALN_SCRATCH, sizeof(int32_t) * 18 * (size_t)W * nwarps);
        ext_out *ext;
        PASTIS_WS(ext, ctx, WS_ALN_PASS1, sizeof(ext_out) * 4 * (size_t)n_pairs);
        prof_begin(ctx, "xd_extend");
        k_xd_ext<<<blocks, ALN_THREADS, 0, st>>>(d_codes, d_offsets, d_pairs, n_pairs, params->k, dmat,
                                                 params->gap_open, params->gap_extend, params->xdrop, gbuf, W,
                                                 flags + 6, ext);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
        prof_begin(ctx, "xd_combine");
        k_xd_combine<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(
            d_codes, d_offsets, d_pairs, n_pairs, params->k, dmat, params->ani_min_pct, params->cov_min_pct, ext,
            d_out, (unsigned long long *)d_cells);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    int herr = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&herr, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    return herr ? PASTIS_ERR_INTERNAL : PASTIS_OK;
}
