// a8-a9: the alignment entry point and the x-drop seed-and-extend (Sec. IV-E, Sec. VI).
// Smith-Waterman lives in sw.cu.
//
// x-drop (XD): from a seed, the seed's score plus two anchored extensions (right of
// the seed, and left of it on the reversed prefixes), each computed antidiagonal by
// antidiagonal by one warp: cells of antidiagonal d+1 are those adjacent to the live
// range of d, a cell dies when H < best - X (best over the earlier antidiagonals),
// and the extension ends when an antidiagonal has no live cell.  Every state carries
// (identities << 16 | matched columns) along the predecessor a traceback would take
// (diagonal > F > E, open > extend), so the end cell holds the path's statistics.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.cuh"

pastis_status sw_align(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets, const uint8_t *d_tcodes,
                       const int64_t *d_toffsets, const pastis_cand *d_pairs, int64_t n_pairs, const pastis_params *p,
                       const int8_t *dmat, int *flags, int lmax, pastis_aln *d_out, int64_t *d_cells,
                       const int64_t *dn, const int *chk);

namespace {

constexpr int NEG = -1000000000;
constexpr int ALN_THREADS = 256;
constexpr int ALN_WARPS = ALN_THREADS / 32;
constexpr int PAD_SCORE = -30000;

__device__ void load_matrix(const int8_t *gmat, int *s_mat) {
    for (int x = threadIdx.x; x < (PASTIS_NSYM + 1) * 32; x += blockDim.x) {
        int a = x / 32, b = x % 32;
        s_mat[x] = (a < PASTIS_NSYM && b < PASTIS_NSYM) ? (int)gmat[a * PASTIS_NSYM + b] : PAD_SCORE;
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
// CARRY = false computes the same scores, ends and cells without the carried statistics
// (res->carry = 0): the first phase of the filter-only mode.
template <bool CARRY>
__device__ void xd_extend_warp(const uint8_t *q, int A, int qs, const uint8_t *t, int B, int ts,
                               const int *s_mat, int o, int e, int X, xd_bufs buf, int W, ext_out *res) {
    const int lane = threadIdx.x & 31;
    int lo[3], hi[3];                       // computed range of the three antidiagonals
    // antidiagonal 0: the anchor
    if (lane == 0) {
        buf.H[0] = 0; buf.E[0] = NEG; buf.F[0] = NEG;
        if constexpr (CARRY) { buf.HC[0] = 0; buf.EC[0] = 0; buf.FC[0] = 0; }
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
                if (eo >= ex) { ev = eo; if constexpr (CARRY) evc = HC1[a]; }
                else { ev = ex; if constexpr (CARRY) evc = EC1[a]; }
                if (ev < NEG) ev = NEG;
            }
            if (a >= 1 && a - 1 >= lo1 && a - 1 <= hi1) {
                const int fo = H1[a - 1] - o, fx = F1[a - 1] - e;
                if (fo >= fx) { fv = fo; if constexpr (CARRY) fvc = HC1[a - 1]; }
                else { fv = fx; if constexpr (CARRY) fvc = FC1[a - 1]; }
                if (fv < NEG) fv = NEG;
            }
            if (a >= 1 && b >= 1 && a - 1 >= lo2 && a - 1 <= hi2) {
                const int hd = H2[a - 1];
                if (hd != NEG) {
                    const int qa = q[(long long)(a - 1) * qs], tb = t[(long long)(b - 1) * ts];
                    dv = hd + s_mat[qa * 32 + tb];
                    if constexpr (CARRY) dvc = HC2[a - 1] + (qa == tb ? 0x10001u : 1u);
                }
            }
            int h = dv;
            uint32_t hc = dvc;
            if (fv > h) { h = fv; hc = fvc; }
            if (ev > h) { h = ev; hc = evc; }
            if (h < best - X) { h = NEG; ev = NEG; fv = NEG; }
            Hd[a] = h; Ed[a] = ev; Fd[a] = fv;
            if constexpr (CARRY) { HCd[a] = hc; ECd[a] = evc; FCd[a] = fvc; }
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
            uint32_t oc = 0u;
            if constexpr (CARRY) oc = __shfl_xor_sync(0xffffffffu, my_bc, x);
            if (ob > my_best || (ob == my_best && oa < my_ba)) { my_best = ob; my_ba = oa; my_bc = oc; }
        }
        __syncwarp();
        if (my_hi < 0) break;
        if (my_best > best) { best = my_best; ba = my_ba; bb = d - my_ba; bc = my_bc; }
        llo = my_lo; lhi = my_hi;
    }
    res->score = best; res->a = ba; res->b = bb; res->carry = CARRY ? bc : 0u; res->cells = cells;
}

// The same extension with the cells indexed by diagonal k = a - b instead of by a.  Along
// an alignment the live cells stay near a few diagonals, so a window of 128 diagonals
// holds them: lane L owns diagonals kbase + 4L .. kbase + 4L + 3 and keeps each one's
// latest H, E, F and carries.  Antidiagonal d has cells only on diagonals of d's parity,
// two per lane; a cell's diagonal predecessor (d-2) is its own diagonal, its E (a, b-1)
// and F (a-1, b) predecessors (d-1) the diagonals k+1 and k-1: in the lane itself except
// one, which one shuffle brings from the next or previous lane.  Cells outside the
// computed range of the definition above are set dead, so the result is the same as
// xd_extend_warp's.  The window moves by whole lanes when the computed range leaves it;
// a range wider than XD_BAND cells returns false (nothing written) and the caller runs
// xd_extend_warp.
constexpr int XD_BAND = 64;                 // cells of one antidiagonal: 32 lanes x 2

struct xd_src { int h, x; uint32_t hc, xc; };   // a predecessor cell: H, E or F, and carries

template <bool CARRY>
__device__ __forceinline__ void xd_cell(int a, int b, int d, int clo, int chi, const uint8_t *q, int qs,
                                        const uint8_t *t, int ts, const int *s_mat, int o, int e, int lim,
                                        const xd_src &se, const xd_src &sf, int &H, int &E, int &F, uint32_t &HC,
                                        uint32_t &EC, uint32_t &FC) {
    int ev = NEG, fv = NEG, h = NEG;
    uint32_t evc = 0u, fvc = 0u, hc = 0u;
    if (a >= clo && a <= chi) {
        if (b >= 1) {
            const int eo = se.h - o, ex = se.x - e;
            if (eo >= ex) { ev = eo; if constexpr (CARRY) evc = se.hc; }
            else { ev = ex; if constexpr (CARRY) evc = se.xc; }
            if (ev < NEG) ev = NEG;
        }
        if (a >= 1) {
            const int fo = sf.h - o, fx = sf.x - e;
            if (fo >= fx) { fv = fo; if constexpr (CARRY) fvc = sf.hc; }
            else { fv = fx; if constexpr (CARRY) fvc = sf.xc; }
            if (fv < NEG) fv = NEG;
        }
        int dv = NEG;
        uint32_t dvc = 0u;
        if (a >= 1 && b >= 1 && H != NEG) {
            const int qa = q[(long long)(a - 1) * qs], tb = t[(long long)(b - 1) * ts];
            dv = H + s_mat[qa * 32 + tb];
            if constexpr (CARRY) dvc = HC + (qa == tb ? 0x10001u : 1u);
        }
        h = dv; hc = dvc;
        if (fv > h) { h = fv; if constexpr (CARRY) hc = fvc; }
        if (ev > h) { h = ev; if constexpr (CARRY) hc = evc; }
        if (h < lim) { h = NEG; ev = NEG; fv = NEG; }
    }
    (void)d;
    H = h; E = ev; F = fv; HC = hc; EC = evc; FC = fvc;
}

template <bool CARRY>
__device__ bool xd_diag_warp(const uint8_t *q, int A, int qs, const uint8_t *t, int B, int ts, const int *s_mat,
                             int o, int e, int X, ext_out *res) {
    const int lane = threadIdx.x & 31;
    int H[4], E[4], F[4];
    uint32_t HC[4], EC[4], FC[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) { H[m] = NEG; E[m] = NEG; F[m] = NEG; HC[m] = 0u; EC[m] = 0u; FC[m] = 0u; }
    int kbase = -64;                        // diagonal 0 (the anchor) at lane 16, m = 0
    if (lane == 16) H[0] = 0;
    int best = 0, ba = 0, bb = 0;
    uint32_t bc = 0;
    long long cells = 1;
    int llo = 0, lhi = 0;
    for (int d = 1; d <= A + B; ++d) {
        const int clo = max(max(llo, d - B), 0);
        const int chi = min(min(lhi + 1, A), d);
        if (clo > chi) break;
        if (chi - clo + 1 > XD_BAND) return false;
        // diagonals of the computed range are [2 clo - d, 2 chi - d]; with their E and F
        // predecessors one further on each side they must lie inside the window
        const int kmin = 2 * clo - d - 1, kmax = 2 * chi - d + 1;
        if (kmin < kbase || kmax > kbase + 127) {
            const int sh = ((kmin + kmax) / 2 - (kbase + 64)) / 4;     // whole lanes, centring the range
            kbase += 4 * sh;
            if (kmin < kbase || kmax > kbase + 127) return false;
            const int src = lane + sh;
            const bool in = (unsigned)src < 32u;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int h = __shfl_sync(0xffffffffu, H[m], src & 31), ee = __shfl_sync(0xffffffffu, E[m], src & 31);
                const int ff = __shfl_sync(0xffffffffu, F[m], src & 31);
                H[m] = in ? h : NEG; E[m] = in ? ee : NEG; F[m] = in ? ff : NEG;
                if constexpr (CARRY) {
                    const uint32_t hc = __shfl_sync(0xffffffffu, HC[m], src & 31);
                    const uint32_t ec = __shfl_sync(0xffffffffu, EC[m], src & 31);
                    const uint32_t fc = __shfl_sync(0xffffffffu, FC[m], src & 31);
                    HC[m] = in ? hc : 0u; EC[m] = in ? ec : 0u; FC[m] = in ? fc : 0u;
                }
            }
        }
        const int lim = best - X;
        const int k0 = kbase + 4 * lane;       // this lane's first diagonal
        int h0, h1, a0;
        uint32_t c0, c1;
        if ((d & 1) == 0) {
            // cells on m = 0 and m = 2; F of m = 0 is the previous lane's m = 3
            xd_src up;
            up.h = __shfl_up_sync(0xffffffffu, H[3], 1); up.x = __shfl_up_sync(0xffffffffu, F[3], 1);
            up.hc = 0u; up.xc = 0u;
            if constexpr (CARRY) {
                up.hc = __shfl_up_sync(0xffffffffu, HC[3], 1); up.xc = __shfl_up_sync(0xffffffffu, FC[3], 1);
            }
            if (lane == 0) { up.h = NEG; up.x = NEG; }
            const xd_src e0{H[1], E[1], HC[1], EC[1]}, e2{H[3], E[3], HC[3], EC[3]};
            const xd_src f2{H[1], F[1], HC[1], FC[1]};
            a0 = (d + k0) >> 1;
            xd_cell<CARRY>(a0, d - a0, d, clo, chi, q, qs, t, ts, s_mat, o, e, lim, e0, up, H[0], E[0], F[0], HC[0], EC[0],
                    FC[0]);
            xd_cell<CARRY>(a0 + 1, d - a0 - 1, d, clo, chi, q, qs, t, ts, s_mat, o, e, lim, e2, f2, H[2], E[2], F[2], HC[2],
                    EC[2], FC[2]);
            h0 = H[0]; h1 = H[2]; c0 = HC[0]; c1 = HC[2];
        } else {
            // cells on m = 1 and m = 3; E of m = 3 is the next lane's m = 0
            xd_src dn;
            dn.h = __shfl_down_sync(0xffffffffu, H[0], 1); dn.x = __shfl_down_sync(0xffffffffu, E[0], 1);
            dn.hc = 0u; dn.xc = 0u;
            if constexpr (CARRY) {
                dn.hc = __shfl_down_sync(0xffffffffu, HC[0], 1); dn.xc = __shfl_down_sync(0xffffffffu, EC[0], 1);
            }
            if (lane == 31) { dn.h = NEG; dn.x = NEG; }
            const xd_src e1{H[2], E[2], HC[2], EC[2]}, f1{H[0], F[0], HC[0], FC[0]};
            const xd_src f3{H[2], F[2], HC[2], FC[2]};
            a0 = (d + k0 + 1) >> 1;
            xd_cell<CARRY>(a0, d - a0, d, clo, chi, q, qs, t, ts, s_mat, o, e, lim, e1, f1, H[1], E[1], F[1], HC[1], EC[1],
                    FC[1]);
            xd_cell<CARRY>(a0 + 1, d - a0 - 1, d, clo, chi, q, qs, t, ts, s_mat, o, e, lim, dn, f3, H[3], E[3], F[3], HC[3],
                    EC[3], FC[3]);
            h0 = H[1]; h1 = H[3]; c0 = HC[1]; c1 = HC[3];
        }
        cells += chi - clo + 1;
        const bool l0 = h0 != NEG, l1 = h1 != NEG;
        const unsigned live = __ballot_sync(0xffffffffu, l0 || l1);
        if (!live) break;
        // the lane's best live cell (the smaller a first) and its live range
        int myh = NEG, mya = 0x7FFFFFFF;
        uint32_t myc = 0u;
        if (l0) { myh = h0; mya = a0; myc = c0; }
        if (l1 && h1 > myh) { myh = h1; mya = a0 + 1; myc = c1; }
        const int toph = __reduce_max_sync(0xffffffffu, myh);
        if (toph > best) {
            const int ta = (int)__reduce_min_sync(0xffffffffu, myh == toph ? (unsigned)mya : 0xFFFFFFFFu);
            if constexpr (CARRY) {
                const unsigned who = __ballot_sync(0xffffffffu, myh == toph && mya == ta);
                bc = __shfl_sync(0xffffffffu, myc, __ffs(who) - 1);
            }
            best = toph; ba = ta; bb = d - ta;
        }
        const int first = __ffs(live) - 1, lastl = 31 - __clz(live);
        const int lo_here = l0 ? a0 : a0 + 1, hi_here = l1 ? a0 + 1 : a0;
        llo = __shfl_sync(0xffffffffu, lo_here, first);
        lhi = __shfl_sync(0xffffffffu, hi_here, lastl);
    }
    res->score = best; res->a = ba; res->b = bb; res->carry = CARRY ? bc : 0u; res->cells = cells;
    return true;
}

// ---------------------------------------------------------------------------------
// The same extensions in 16-bit lanes, several per warp, with or without the carried
// statistics.
//
// The diagonal window of xd_diag_warp (128 diagonals, at most 64 computed cells per
// antidiagonal) is split over G = 32 / R lanes, so a warp runs R extensions side by
// side, each in a segment of G lanes.  Lane s of a segment owns the 4R diagonals
// kbase + 4R s .. kbase + 4R s + 4R - 1; on antidiagonal d it computes the 2R cells of
// d's parity, in R registers of two signed 16-bit halves: register r of the even set
// holds the diagonals at offsets 4r and 4r + 2, of the odd set 4r + 1 and 4r + 3.  A
// lane's cells of one antidiagonal are consecutive rows a0 .. a0 + 2R - 1, so their
// query and target residues are windows that slide by one residue every second
// antidiagonal; the windows hold each residue as its offset into a score table of
// which every lane of the warp has its own copy in its own shared-memory bank.  Per
// register and antidiagonal the recurrence is the packed one of the Smith-Waterman
// pass 1 without the floor at 0: E and F as __viaddmax_s16x2, the diagonal as
// __vadd2, H as __vimax3_s16x2.  The x-drop test (H >= best - X) and the computed range
// [clo, chi] become a per-half mask by clamps alone: min(max(H, lim - 1), lim) - lim
// is -1 exactly where H < lim, min(row - clo, chi - row) is negative exactly outside
// the range, and the mask selects the dead value.
//
// Dead cells hold XD16_NEG in H, E and F.  Live values lie in [best - X - o - e, best
// + the largest substitution score], values derived from dead ones in [XD16_NEG - o -
// e, XD16_NEG + 63], and every one of them is pruned (XD16_NEG + 63 < -X), so no sum
// wraps when X, the best score and o + e stay within the bounds checked below; an
// extension outside them, or whose computed range outgrows the window, is listed for
// the 32-bit kernel, which computes it from the start.
//
// Every lane runs every step, an odd antidiagonal and an even one per turn of one
// loop, so the segments' parities agree and the packed sources need no per-segment
// branch; a segment whose extension has ended computes on empty ranges and writes
// nothing until it takes the next extension at the top of the loop.  The end cell is
// found once per extension: the step that raises the best score keeps a copy of its
// H registers, and the first row holding the best is read from that copy at the end.
//
// The carried statistics (identities and aligned columns along the path a traceback
// from the cell would take, Sec. IV-E) are one 32-bit word per cell beside H, E and F,
// for both parities.  A cell's words follow its winning predecessor: E and F take H's
// (gap open) unless the extension wins outright, H takes the diagonal's plus one
// column (and one identity when the residues match) unless F, then E, is strictly
// larger.  Which candidate won is read off the packed results: a half of max(x, y)
// equals x's exactly when x won or tied.  The score table then holds each score's byte
// and the match bit (q == t) above it; the scores are sign-extended from the bytes.
// ---------------------------------------------------------------------------------
constexpr int XD16_NEG = -32512;                 // 0x8100
constexpr uint32_t XD16_NEG2 = (uint32_t)(XD16_NEG & 0xffff) * 0x10001u;   // 0x81008100
constexpr int XD16_LIM = 30000;                  // bound on X and on an extension's best score
// Score table, int16: byte offset q * 1536 + (t >> 1) * 128 + (t & 1) * 2 + 4 * lane holds
// s(q, t) (with carries: the byte of s(q, t), then [q == t]) for every lane, so lane L
// always reads bank L.
constexpr int XD16_TAB = PASTIS_NSYM * PASTIS_NSYM * 32;   // entries
constexpr uint32_t XD16_QOFF = PASTIS_NSYM / 2 * 128;      // bytes per query residue

// Whether the 16-bit kernel may run an x-drop with these penalties at all.
static inline bool xd16_params_fit(int o, int e, int X) { return o <= 128 && e <= 128 && X <= XD16_LIM; }

__device__ __forceinline__ uint32_t xd16_pk(int v) { return __byte_perm((uint32_t)v, 0u, 0x1010); }

// The low bytes of a and b as two signed 16-bit halves: prmt in its default mode copies a
// byte where a selector nibble has bit 3 clear and replicates its sign bit where it is set.
__device__ __forceinline__ uint32_t xd16_sext_lo_bytes(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, 0xC480;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// Live bits of four cells in row order from the dead masks of two registers (halves of
// 0xffff or 0): the high byte of each half, gathered in row order, then its top bit
// moved to bit j by one multiply (the partial products below bit 28 never carry into it).
__device__ __forceinline__ uint32_t xd16_live4(uint32_t dm0, uint32_t dm1) {
    const uint32_t x = ~__byte_perm(dm0, dm1, 0x7531) & 0x80808080u;
    return (x * 0x00204081u) >> 28;
}

template <int R, bool C>
struct xd16_ext {
    uint32_t H[2][R], E[2][R], F[2][R];          // [parity of the diagonals][register]
    uint32_t QW[R], TW[R];                       // cells 2r (low half), 2r + 1: table offsets of q and t
    uint32_t HS[R];                              // H of the antidiagonal sd that last raised best
    // C: the carried statistics (identities << 16 | columns) of H, E and F, one word per
    // cell [parity][register][half], and those of HS
    uint32_t HC[2][C ? R : 1][2], EC[2][C ? R : 1][2], FC[2][C ? R : 1][2], HSC[C ? R : 1][2];
    const uint8_t *q, *t;
    int st, A, B;                                // A = B = 0 while the segment has no extension
    int d, best, sd, sa0, llo, lhi, kbase;
    long long cells;
    int64_t task;
    bool active;
};

// Table offset of query residue idx (0 outside the sequence), and of target residue idx
// plus this lane's column.
template <int R, bool C>
__device__ __forceinline__ uint32_t xd16_qoff(const xd16_ext<R, C> &x, int idx) {
    return (unsigned)idx < (unsigned)x.A ? (uint32_t)x.q[(long long)idx * x.st] * XD16_QOFF : 0u;
}
template <int R, bool C>
__device__ __forceinline__ uint32_t xd16_toff(const xd16_ext<R, C> &x, int idx, uint32_t lane4) {
    uint32_t c = (unsigned)idx < (unsigned)x.B ? (uint32_t)x.t[(long long)idx * x.st] : 0u;
    return (c >> 1) * 128u + (c & 1u) * 2u + lane4;
}

// The windows for antidiagonal d whose first row in this lane is a0: cell j has query
// residue a0 + j - 1 and target residue d - a0 - j - 1.
template <int R, bool C>
__device__ __forceinline__ void xd16_load_windows(xd16_ext<R, C> &x, int d, int a0, uint32_t lane4) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        x.QW[r] = xd16_qoff(x, a0 + 2 * r - 1) | (xd16_qoff(x, a0 + 2 * r) << 16);
        x.TW[r] = xd16_toff(x, d - a0 - 2 * r - 1, lane4) | (xd16_toff(x, d - a0 - 2 * r - 2, lane4) << 16);
    }
}

// One antidiagonal (d = x.d + 1, of parity PAR) of the segment's extension, run by every
// lane of the warp.
template <int R, bool C, int PAR>
__device__ __forceinline__ void xd16_step(xd16_ext<R, C> &x, int ls, unsigned smask, int sbase, const char *tab,
                                          uint32_t lane4, uint32_t o2, uint32_t ne2, int X, ext_out *out,
                                          uint32_t *ovf_list, uint32_t *ovf_n) {
    constexpr int G = 32 / R, WD = 4 * R, NC = 2 * R;
    constexpr int P = PAR, Q = 1 - PAR;
    const int d = x.d + 1;
    const int clo = max(max(x.llo, d - x.B), 0);
    const int chi = min(min(x.lhi + 1, x.A), d);
    const bool empty = clo > chi;                        // the extension ended (d > A + B included)
    bool defer = !empty && chi - clo + 1 > G * NC;
    // the computed range's diagonals, with their E and F predecessors, inside the window
    const int kmin = 2 * clo - d - 1, kmax = 2 * chi - d + 1;
    const bool move = !empty && !defer && (kmin < x.kbase || kmax > x.kbase + 127);
    int a0 = (d + x.kbase + WD * ls + P) >> 1;          // this lane's first row on d
    if (P == 1) {        // rows moved on by one: a new last query residue
#pragma unroll
        for (int r = 0; r < R; ++r)
            x.QW[r] = __byte_perm(x.QW[r], r == R - 1 ? xd16_qoff(x, a0 + NC - 2) : x.QW[r + 1], 0x5432);
    } else {             // columns moved on by one: a new first target residue
#pragma unroll
        for (int r = R - 1; r >= 0; --r)
            x.TW[r] = __byte_perm(r == 0 ? xd16_toff(x, d - a0 - 1, lane4) << 16 : x.TW[r - 1], x.TW[r], 0x5432);
    }
    if (__any_sync(0xffffffffu, move)) {
        if (move) {
            const int sh = ((kmin + kmax) / 2 - (x.kbase + 64)) / WD;      // whole lanes, centring the range
            x.kbase += WD * sh;
            if (kmin < x.kbase || kmax > x.kbase + 127) {
                defer = true;
            } else {
                const int src = ls + sh;
                const bool in = (unsigned)src < (unsigned)G;
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const uint32_t h = __shfl_sync(smask, x.H[p][r], src & (G - 1), G);
                        const uint32_t ee = __shfl_sync(smask, x.E[p][r], src & (G - 1), G);
                        const uint32_t ff = __shfl_sync(smask, x.F[p][r], src & (G - 1), G);
                        x.H[p][r] = in ? h : XD16_NEG2;
                        x.E[p][r] = in ? ee : XD16_NEG2;
                        x.F[p][r] = in ? ff : XD16_NEG2;
                        if constexpr (C) {
#pragma unroll
                            for (int hf = 0; hf < 2; ++hf) {
                                const uint32_t hc = __shfl_sync(smask, x.HC[p][r][hf], src & (G - 1), G);
                                const uint32_t ec = __shfl_sync(smask, x.EC[p][r][hf], src & (G - 1), G);
                                const uint32_t fc = __shfl_sync(smask, x.FC[p][r][hf], src & (G - 1), G);
                                x.HC[p][r][hf] = in ? hc : 0u;
                                x.EC[p][r][hf] = in ? ec : 0u;
                                x.FC[p][r][hf] = in ? fc : 0u;
                            }
                        }
                    }
                a0 = (d + x.kbase + WD * ls + P) >> 1;
                xd16_load_windows(x, d, a0, lane4);
            }
        }
    }
    const int lim = x.best - X;
    const uint32_t lim2 = xd16_pk(lim), limm2 = __vsub2(lim2, 0x00010001u);
    const uint32_t span2 = xd16_pk(chi - clo), rb2 = xd16_pk(a0 - clo);
    // the sources on d - 1 that cross a lane boundary
    uint32_t bh, bx, bhc = 0u, bxc = 0u;
    if (P == 0) {        // F of the first cell: the previous lane's last odd diagonal
        bh = __shfl_up_sync(0xffffffffu, x.H[Q][R - 1], 1, G);
        bx = __shfl_up_sync(0xffffffffu, x.F[Q][R - 1], 1, G);
        if constexpr (C) {
            bhc = __shfl_up_sync(0xffffffffu, x.HC[Q][R - 1][1], 1, G);
            bxc = __shfl_up_sync(0xffffffffu, x.FC[Q][R - 1][1], 1, G);
        }
        if (ls == 0) { bh = XD16_NEG2; bx = XD16_NEG2; }
    } else {             // E of the last cell: the next lane's first even diagonal
        bh = __shfl_down_sync(0xffffffffu, x.H[Q][0], 1, G);
        bx = __shfl_down_sync(0xffffffffu, x.E[Q][0], 1, G);
        if constexpr (C) {
            bhc = __shfl_down_sync(0xffffffffu, x.HC[Q][0][0], 1, G);
            bxc = __shfl_down_sync(0xffffffffu, x.EC[Q][0][0], 1, G);
        }
        if (ls == G - 1) { bh = XD16_NEG2; bx = XD16_NEG2; }
    }
    uint32_t dmk[R];                             // dead masks, for the live bits below
    uint32_t hmax = XD16_NEG2;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        uint32_t eh, ex, fh, fx;
        if (P == 0) {
            eh = x.H[Q][r]; ex = x.E[Q][r];
            fh = __byte_perm(r == 0 ? bh : x.H[Q][r - 1], x.H[Q][r], 0x5432);
            fx = __byte_perm(r == 0 ? bx : x.F[Q][r - 1], x.F[Q][r], 0x5432);
        } else {
            fh = x.H[Q][r]; fx = x.F[Q][r];
            eh = __byte_perm(x.H[Q][r], r == R - 1 ? bh : x.H[Q][r + 1], 0x5432);
            ex = __byte_perm(x.E[Q][r], r == R - 1 ? bx : x.E[Q][r + 1], 0x5432);
        }
        const uint32_t eo = __vsub2(eh, o2), fo = __vsub2(fh, o2);
        const uint32_t en = __viaddmax_s16x2(ex, ne2, eo);
        const uint32_t fn = __viaddmax_s16x2(fx, ne2, fo);
        // substitution scores of rows a0 + 2r and a0 + 2r + 1 from this lane's table column
        const uint32_t ix = x.QW[r] + x.TW[r];
        const uint32_t s0 = *(const uint16_t *)(tab + (ix & 0xffffu));
        const uint32_t s1 = *(const uint16_t *)(tab + (ix >> 16));
        // with carries an entry is the score's byte, then [q == t]: the scores sign-extended
        const uint32_t dg = __vadd2(x.H[P][r], C ? xd16_sext_lo_bytes(s0, s1) : __byte_perm(s0, s1, 0x5410));
        const uint32_t hn = __vimax3_s16x2(dg, en, fn);
        if constexpr (C) {
            // each cell's carries along the predecessor a traceback takes: E and F from H
            // (the gap opens) on ties, H from the diagonal, then from F, then from E; a
            // packed result equals the candidate it came from
            const uint32_t xe = en ^ eo, xf = fn ^ fo, xdg = dg ^ hn, xfh = fn ^ hn;
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                auto zero = [hf](uint32_t v) { return hf ? (v >> 16) == 0u : (v & 0xffffu) == 0u; };
                uint32_t ehc, exc, fhc, fxc;
                if (P == 0) {
                    ehc = x.HC[Q][r][hf]; exc = x.EC[Q][r][hf];
                    fhc = hf ? x.HC[Q][r][0] : (r == 0 ? bhc : x.HC[Q][r > 0 ? r - 1 : 0][1]);
                    fxc = hf ? x.FC[Q][r][0] : (r == 0 ? bxc : x.FC[Q][r > 0 ? r - 1 : 0][1]);
                } else {
                    fhc = x.HC[Q][r][hf]; fxc = x.FC[Q][r][hf];
                    ehc = hf ? (r == R - 1 ? bhc : x.HC[Q][r < R - 1 ? r + 1 : 0][0]) : x.HC[Q][r][1];
                    exc = hf ? (r == R - 1 ? bxc : x.EC[Q][r < R - 1 ? r + 1 : 0][0]) : x.EC[Q][r][1];
                }
                const uint32_t evc = zero(xe) ? ehc : exc;
                const uint32_t fvc = zero(xf) ? fhc : fxc;
                const uint32_t dvc = x.HC[P][r][hf] + 1u + (((hf ? s1 : s0) >> 8) << 16);
                x.HC[P][r][hf] = zero(xdg) ? dvc : (zero(xfh) ? fvc : evc);
                x.EC[P][r][hf] = evc;
                x.FC[P][r][hf] = fvc;
            }
        }
        // dead halves: H < lim, or the row outside [clo, chi]
        const uint32_t rr = __vadd2(rb2, (uint32_t)((2 * r) | ((2 * r + 1) << 16)));
        const uint32_t w = __vmins2(rr, __vsub2(span2, rr));
        const uint32_t d1 = __vsub2(__vmins2(__vmaxs2(hn, limm2), lim2), lim2);
        const uint32_t dm = __vmins2(d1, __vmaxs2(w, 0xffffffffu));
        x.H[P][r] = (hn & ~dm) | (XD16_NEG2 & dm);
        x.E[P][r] = (en & ~dm) | (XD16_NEG2 & dm);
        x.F[P][r] = (fn & ~dm) | (XD16_NEG2 & dm);
        dmk[r] = dm;
        hmax = __vmaxs2(hmax, x.H[P][r]);
    }
    // live cells of this lane, bit j = row a0 + j
    uint32_t lb;
    if (R == 1) {
        const uint32_t y = ~dmk[0] & 0x80008000u;
        lb = ((y >> 15) & 1u) | (y >> 30);
    } else {
        lb = xd16_live4(dmk[0], dmk[R > 1 ? 1 : 0]);
        if (R == 4) lb |= xd16_live4(dmk[R > 2 ? 2 : 0], dmk[R > 3 ? 3 : 0]) << 4;
    }
    x.cells += empty ? 0 : chi - clo + 1;
    x.d = d;
    const unsigned bal = (__ballot_sync(0xffffffffu, lb != 0u) >> sbase) & (G == 32 ? 0xffffffffu : ((1u << G) - 1u));
    const int myh = max((int)(short)(hmax & 0xffffu), (int)hmax >> 16);
    // the segment's maximum by a butterfly of full-warp shuffles (a reduction with a
    // per-segment member mask runs once per distinct mask)
    int toph = myh;
#pragma unroll
    for (int m = G / 2; m > 0; m >>= 1) toph = max(toph, __shfl_xor_sync(0xffffffffu, toph, m, G));
    const bool raise = !empty && !defer && toph > x.best;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        x.HS[r] = raise ? x.H[P][r] : x.HS[r];
        if constexpr (C) {
            x.HSC[r][0] = raise ? x.HC[P][r][0] : x.HSC[r][0];
            x.HSC[r][1] = raise ? x.HC[P][r][1] : x.HSC[r][1];
        }
    }
    x.sa0 = raise ? a0 : x.sa0;
    x.sd = raise ? d : x.sd;
    x.best = raise ? toph : x.best;
    const int first = __ffs(bal) - 1, last = 31 - __clz(bal);
    x.llo = __shfl_sync(0xffffffffu, a0 + __ffs(lb) - 1, first & (G - 1), G);
    x.lhi = __shfl_sync(0xffffffffu, a0 + 31 - __clz(lb), last & (G - 1), G);
    // the end of the extension, or its hand-over to the 32-bit kernel
    const bool stop = x.active && (defer || empty || bal == 0u);
    if (__any_sync(0xffffffffu, stop)) {
        if (stop) {
            if (defer) {
                if (ls == 0) ovf_list[atomicAdd(ovf_n, 1u)] = (uint32_t)x.task;
            } else {
                // the first row holding best on the antidiagonal that raised it last
                unsigned mya = 0xFFFFFFFFu;
                uint32_t myc = 0u;
#pragma unroll
                for (int j = NC - 1; j >= 0; --j) {
                    const uint32_t v = x.HS[j >> 1];
                    if (((j & 1) ? (int)v >> 16 : (int)(short)(v & 0xffffu)) == x.best) {
                        mya = (unsigned)(x.sa0 + j);
                        if constexpr (C) myc = x.HSC[j >> 1][j & 1];
                    }
                }
                const int ta = (int)__reduce_min_sync(smask, mya);
                uint32_t carry = 0u;
                if constexpr (C) {
                    // the carries of the lane that holds the end cell
                    const unsigned who = __ballot_sync(smask, mya == (unsigned)ta);
                    carry = __shfl_sync(smask, myc, (__ffs(who) - 1) & (G - 1), G);
                }
                if (ls == 0) {
                    ext_out res;
                    res.score = x.best;
                    res.a = x.best > 0 ? ta : 0;
                    res.b = x.best > 0 ? x.sd - ta : 0;
                    res.carry = x.best > 0 ? carry : 0u;
                    res.cells = x.cells;
                    out[x.task] = res;
                }
            }
            x.active = false;
            x.A = 0;
            x.B = 0;
        }
    }
}

// Extensions in 16-bit lanes: every task (4 p + 2 seed + left; with a task list the
// listed ones, *d_ntask of them) whose extension fits gets its score, end and cells, and
// with C its carried statistics; the others are listed in ovf_list[*ovf_n] for k_xd_ext.
// smax = the largest substitution score; s_tab = the CTA's score table.
template <int R, bool C>
__device__ __forceinline__ void xd16_run(const uint8_t *qcodes, const int64_t *qoffsets, const uint8_t *tcodes,
                                         const int64_t *toffsets, const pastis_cand *pairs, int64_t n_pairs, int k,
                                         const int8_t *gmat, int o, int e, int X, int smax, int *next_task,
                                         ext_out *out, uint32_t *ovf_list, uint32_t *ovf_n,
                                         const uint32_t *task_list, const uint32_t *d_ntask, const int64_t *dn,
                                         const int *chk, uint16_t *s_tab) {
    constexpr int G = 32 / R, WD = 4 * R;
    if (dn) n_pairs = *dn;
    if (chk && (chk[0] | chk[1])) return;
    for (int i = threadIdx.x; i < XD16_TAB; i += blockDim.x) {
        // i = q * 768 + (t >> 1) * 64 + lane * 2 + (t & 1)
        const int q = i / 768, t = ((i % 768) >> 6) * 2 + (i & 1);
        const int v = gmat[q * PASTIS_NSYM + t];
        s_tab[i] = C ? (uint16_t)((v & 0xff) | (q == t ? 0x100 : 0)) : (uint16_t)v;
    }
    __syncthreads();
    const char *tab = (const char *)s_tab;
    const int lane = threadIdx.x & 31;
    const uint32_t lane4 = 4u * (uint32_t)lane;
    const int seg = lane / G, ls = lane % G, sbase = seg * G;
    const unsigned smask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << sbase);
    const uint32_t o2 = xd16_pk(o), ne2 = xd16_pk(-e);
    const int64_t ntask = task_list ? (int64_t)*d_ntask : n_pairs * 4;
    xd16_ext<R, C> x;
    x.active = false;
    x.A = 0; x.B = 0; x.d = 0; x.best = 0; x.sd = 0; x.sa0 = 0; x.llo = 0; x.lhi = 0; x.kbase = -64; x.cells = 0;
    x.task = 0; x.st = 1; x.q = qcodes; x.t = tcodes;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        x.H[0][r] = x.H[1][r] = x.E[0][r] = x.E[1][r] = x.F[0][r] = x.F[1][r] = XD16_NEG2;
        x.QW[r] = 0u; x.TW[r] = lane4 | (lane4 << 16); x.HS[r] = XD16_NEG2;
        if constexpr (C)
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                x.HC[0][r][hf] = x.HC[1][r][hf] = x.EC[0][r][hf] = x.EC[1][r][hf] = 0u;
                x.FC[0][r][hf] = x.FC[1][r][hf] = x.HSC[r][hf] = 0u;
            }
    }
    bool exhausted = false;
    for (;;) {
        if (__any_sync(0xffffffffu, !x.active && !exhausted)) {
            while (!x.active && !exhausted) {
                unsigned long long slot = 0;
                if (ls == 0) slot = atomicAdd((unsigned long long *)next_task, 1ull);
                slot = __shfl_sync(smask, slot, 0, G);
                if ((int64_t)slot >= ntask) { exhausted = true; break; }
                x.task = task_list ? (int64_t)task_list[slot] : (int64_t)slot;
                const int64_t p = x.task >> 2;
                const int seed = (int)((x.task >> 1) & 1), left = (int)(x.task & 1);
                const pastis_cand c = pairs[p];
                if (!(seed == 0 || (c.count >= 2 && c.qpos[1] != 0xFFFF))) {
                    if (ls == 0) {
                        ext_out r;
                        r.score = 0; r.a = 0; r.b = 0; r.carry = 0u; r.cells = 0;
                        out[x.task] = r;
                    }
                    continue;
                }
                const int64_t qo = qoffsets[c.i], to = toffsets[c.j];
                const int lq = (int)(qoffsets[c.i + 1] - qo), lt = (int)(toffsets[c.j + 1] - to);
                const int pi = c.qpos[seed], pj = c.tpos[seed];
                const int A = left ? pi : lq - pi - k, B = left ? pj : lt - pj - k;
                if (A < 1 || B < 1 || smax * min(A, B) > XD16_LIM) {
                    if (ls == 0) ovf_list[atomicAdd(ovf_n, 1u)] = (uint32_t)x.task;
                    continue;
                }
                x.q = left ? qcodes + qo + pi - 1 : qcodes + qo + pi + k;
                x.t = left ? tcodes + to + pj - 1 : tcodes + to + pj + k;
                x.A = A; x.B = B; x.st = left ? -1 : 1;
                // antidiagonal 0: the anchor, diagonal 0 = the low half of lane 64 / 4R's
                // first even register
                x.kbase = -64;
#pragma unroll
                for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        x.H[pp][r] = XD16_NEG2; x.E[pp][r] = XD16_NEG2; x.F[pp][r] = XD16_NEG2;
                        if constexpr (C)
#pragma unroll
                            for (int hf = 0; hf < 2; ++hf) {
                                x.HC[pp][r][hf] = 0u; x.EC[pp][r][hf] = 0u; x.FC[pp][r][hf] = 0u;
                            }
                    }
                if (ls == 64 / WD) x.H[0][0] = XD16_NEG2 & 0xffff0000u;
                x.d = 0; x.best = 0; x.sd = 0; x.sa0 = 0; x.llo = 0; x.lhi = 0; x.cells = 1;
                xd16_load_windows(x, 0, (x.kbase + WD * ls) >> 1, lane4);
                x.active = true;
            }
        }
        if (__all_sync(0xffffffffu, exhausted)) break;
        xd16_step<R, C, 1>(x, ls, smask, sbase, tab, lane4, o2, ne2, X, out, ovf_list, ovf_n);
        xd16_step<R, C, 0>(x, ls, smask, sbase, tab, lane4, o2, ne2, X, out, ovf_list, ovf_n);
    }
}


#define XD16_PARAMS                                                                                         \
    const uint8_t *qcodes, const int64_t *qoffsets, const uint8_t *tcodes, const int64_t *toffsets,         \
        const pastis_cand *pairs, int64_t n_pairs, int k, const int8_t *gmat, int o, int e, int X, int smax, \
        int *next_task, ext_out *out, uint32_t *ovf_list, uint32_t *ovf_n, const uint32_t *task_list,       \
        const uint32_t *d_ntask, const int64_t *dn, const int *chk
#define XD16_ARGS                                                                                        \
    qcodes, qoffsets, tcodes, toffsets, pairs, n_pairs, k, gmat, o, e, X, smax, next_task, out, ovf_list, \
        ovf_n, task_list, d_ntask, dn, chk

// Without carries: the filter-only mode's first phase (at most 79 registers: three CTAs
// per SM).
template <int R>
__global__ void __launch_bounds__(ALN_THREADS) k_xd_ext16(XD16_PARAMS) {
    __shared__ uint16_t s_tab[XD16_TAB];
    xd16_run<R, false>(XD16_ARGS, s_tab);
}

// With carries: the filter-only mode's second phase (over its task list) and PASTIS_XD.
// Held to two CTAs per SM: with four extensions per warp the words take 150 registers
// unbounded (one CTA), 128 with a few spilled, and the second occupancy pays more than
// the spills cost.
template <int R>
__global__ void __launch_bounds__(ALN_THREADS, 2) k_xd_ext16_carry(XD16_PARAMS) {
    __shared__ uint16_t s_tab[XD16_TAB];
    xd16_run<R, true>(XD16_ARGS, s_tab);
}
#undef XD16_PARAMS
#undef XD16_ARGS

// Extension tasks: task = 4 p + 2 seed + left.  With a task list the kernel runs only
// the listed tasks (*d_ntask of them): the second phase of the filter-only mode.
template <bool CARRY>
__global__ void __launch_bounds__(ALN_THREADS) k_xd_ext(const uint8_t *qcodes, const int64_t *qoffsets,
                                                        const uint8_t *tcodes, const int64_t *toffsets,
                                                        const pastis_cand *pairs, int64_t n_pairs, int k,
                                                        const int8_t *gmat, int o, int e, int X, int32_t *gbuf,
                                                        int W, int *next_task, ext_out *out,
                                                        const uint32_t *task_list, const uint32_t *d_ntask,
                                                        const int64_t *dn, const int *chk) {
    if (dn) n_pairs = *dn;                       // captured launches: count in device memory
    if (chk && (chk[0] | chk[1])) return;        // ... and nothing on bad input
    __shared__ int s_mat[(PASTIS_NSYM + 1) * 32];
    load_matrix(gmat, s_mat);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * ALN_WARPS + (threadIdx.x >> 5);
    xd_bufs buf;
    int32_t *base = gbuf + (size_t)gw * 18 * W;
    buf.H = base; buf.E = base + 3 * W; buf.F = base + 6 * W;
    buf.HC = (uint32_t *)(base + 9 * W); buf.EC = (uint32_t *)(base + 12 * W); buf.FC = (uint32_t *)(base + 15 * W);
    const int64_t ntask = task_list ? (int64_t)*d_ntask : n_pairs * 4;
    for (;;) {
        int64_t slot = 0;
        if (lane == 0) slot = atomicAdd((unsigned long long *)next_task, 1ull);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= ntask) break;
        const int64_t task = task_list ? (int64_t)task_list[slot] : slot;
        const int64_t p = task >> 2;
        const int seed = (int)((task >> 1) & 1), left = (int)(task & 1);
        const pastis_cand c = pairs[p];
        ext_out r;
        r.score = 0; r.a = 0; r.b = 0; r.carry = 0; r.cells = 0;
        const bool has = seed == 0 || (c.count >= 2 && c.qpos[1] != 0xFFFF);
        if (has) {
            const int64_t qo = qoffsets[c.i], to = toffsets[c.j];
            const int lq = (int)(qoffsets[c.i + 1] - qo), lt = (int)(toffsets[c.j + 1] - to);
            const int pi = c.qpos[seed], pj = c.tpos[seed];
            const uint8_t *qa = left ? qcodes + qo + pi - 1 : qcodes + qo + pi + k;
            const uint8_t *ta = left ? tcodes + to + pj - 1 : tcodes + to + pj + k;
            const int A = left ? pi : lq - pi - k, B = left ? pj : lt - pj - k, st = left ? -1 : 1;
            if (!xd_diag_warp<CARRY>(qa, A, st, ta, B, st, s_mat, o, e, X, &r))
                xd_extend_warp<CARRY>(qa, A, st, ta, B, st, s_mat, o, e, X, buf, W, &r);
        }
        if (lane == 0) out[task] = r;
        __syncwarp();
    }
}

// The filter-only mode between its phases: a seed whose alignment (spans known from the
// extension ends alone) leaves less than the coverage bound on the shorter sequence
// cannot pass, so its extensions need no carried statistics; the others (both
// directions of a seed that covers enough) are flagged for the second phase.  Zero past
// the batch, so a scan over the capacity counts the batch's tasks.
__global__ void k_xd_mark(const int64_t *qoffsets, const int64_t *toffsets, const pastis_cand *pairs, int64_t n,
                          int k, int cov, const ext_out *ext, uint32_t *need, const int64_t *dn, const int *chk) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    uint32_t f[2] = {0u, 0u};
    if (!(dn && p >= *dn) && !(chk && (chk[0] | chk[1]))) {
        const pastis_cand c = pairs[p];
        const int lq = (int)(qoffsets[c.i + 1] - qoffsets[c.i]), lt = (int)(toffsets[c.j + 1] - toffsets[c.j]);
        const int ns = (c.count >= 2 && c.qpos[1] != 0xFFFF) ? 2 : 1;
        for (int s = 0; s < ns; ++s) {
            const ext_out R = ext[p * 4 + s * 2 + 0], L = ext[p * 4 + s * 2 + 1];
            const int span = lq <= lt ? L.a + k + R.a : L.b + k + R.b;
            f[s] = 100 * span >= cov * min(lq, lt) ? 1u : 0u;
        }
    }
    need[p * 4 + 0] = f[0]; need[p * 4 + 1] = f[0];
    need[p * 4 + 2] = f[1]; need[p * 4 + 3] = f[1];
}

// The flagged tasks in order, and their count after them (list[n4]).
__global__ void k_xd_tasks(const uint32_t *need, const uint32_t *off, int64_t n4, uint32_t *list) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n4) return;
    if (need[t]) list[off[t]] = (uint32_t)t;
    if (t == n4 - 1) list[n4] = off[t] + need[t];
}

__global__ void k_xd_combine(const uint8_t *qcodes, const int64_t *qoffsets, const uint8_t *tcodes,
                             const int64_t *toffsets, const pastis_cand *pairs,
                             int64_t n_pairs, int k, const int8_t *gmat, int ani, int cov, int filtered,
                             const ext_out *ext, pastis_aln *out, unsigned long long *cells, const int64_t *dn,
                             const int *chk) {
    if (dn) n_pairs = *dn;
    if (chk && (chk[0] | chk[1])) return;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long my = 0;
    if (p < n_pairs) {
        const pastis_cand c = pairs[p];
        const int64_t qo = qoffsets[c.i], to = toffsets[c.j];
        const int lq = (int)(qoffsets[c.i + 1] - qo), lt = (int)(toffsets[c.j + 1] - to);
        const int ns = (c.count >= 2 && c.qpos[1] != 0xFFFF) ? 2 : 1;
        pastis_aln best;
        bool best_ok = false;
        for (int s = 0; s < ns; ++s) {
            const ext_out R = ext[p * 4 + s * 2 + 0], L = ext[p * 4 + s * 2 + 1];
            const int pi = c.qpos[s], pj = c.tpos[s];
            int seed = 0, sid = 0;
            for (int x = 0; x < k; ++x) {
                const int a = qcodes[qo + pi + x], b = tcodes[to + pj + x];
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
        // the filter-only mode: a pair that fails keeps its score and end (a seed that
        // failed the coverage test has no carried statistics)
        if (filtered && !best_ok) { best.qb = best.tb = 0; best.ident = best.cols = 0; }
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

__global__ void k_check_codes(const uint8_t *codes, int64_t n, int *bad, const int64_t *dn) {
    if (dn) n = *dn;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        if (codes[x] >= PASTIS_NSYM) *bad = 1;
}

__global__ void k_check_pairs(const pastis_cand *pairs, int64_t n_pairs, const int64_t *qoffsets, int32_t n_q,
                              const int64_t *toffsets, int32_t n_t, int k, int xd, int *bad, const int64_t *dc) {
    if (dc) { n_pairs = dc[0]; n_q = (int32_t)dc[2]; }
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const pastis_cand c = pairs[p];
    if (c.i < 0 || c.j < 0 || c.i >= n_q || c.j >= n_t) { *bad = 1; return; }
    if (!xd) return;
    const int lq = (int)(qoffsets[c.i + 1] - qoffsets[c.i]), lt = (int)(toffsets[c.j + 1] - toffsets[c.j]);
    const int ns = (c.count >= 2 && c.qpos[1] != 0xFFFF) ? 2 : 1;
    for (int s = 0; s < ns; ++s)
        if ((int)c.qpos[s] + k > lq || (int)c.tpos[s] + k > lt) *bad = 1;
}

}  // namespace

// A captured launch sequence (the plan's graph): counts in device memory, sizes at
// the plan's capacities, no host synchronisation inside.
struct align_graph {
    const int64_t *dc;     // [0] pairs, [1] query residues, [2] queries
    int lmax;              // the longest sequence the plan admits
    int64_t qres_cap;      // capacity of the query residues
};

// The arguments of k_xd_ext16 / k_xd_ext16_carry that do not change between their launches.
struct xd16_args {
    const uint8_t *qcodes;
    const int64_t *qoffsets;
    const uint8_t *tcodes;
    const int64_t *toffsets;
    const pastis_cand *pairs;
    int64_t n_pairs;
    int k;
    const int8_t *gmat;
    int o, e, X, smax;
    ext_out *out;
    const int64_t *dn;
    const int *chk;
};

template <int R, bool C>
static void launch_xd16_r(pastis_ctx *ctx, const xd16_args &a, int *next_task, uint32_t *ovf_list, uint32_t *ovf_n,
                          const uint32_t *task_list, const uint32_t *d_ntask) {
    int per_sm = 1;
    auto kern = C ? k_xd_ext16_carry<R> : k_xd_ext16<R>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, ALN_THREADS, 0);
    kern<<<ctx->sm_count * std::max(per_sm, 1), ALN_THREADS, 0, ctx->stream>>>(
        a.qcodes, a.qoffsets, a.tcodes, a.toffsets, a.pairs, a.n_pairs, a.k, a.gmat, a.o, a.e, a.X, a.smax, next_task,
        a.out, ovf_list, ovf_n, task_list, d_ntask, a.dn, a.chk);
}

// k_xd_ext16 (C: k_xd_ext16_carry) with per_warp (1, 2 or 4) extensions per warp, one CTA
// per resident slot.
template <bool C>
static void launch_xd16(pastis_ctx *ctx, int per_warp, const xd16_args &a, int *next_task, uint32_t *ovf_list,
                        uint32_t *ovf_n, const uint32_t *task_list, const uint32_t *d_ntask) {
    if (per_warp == 1) launch_xd16_r<1, C>(ctx, a, next_task, ovf_list, ovf_n, task_list, d_ntask);
    else if (per_warp == 2) launch_xd16_r<2, C>(ctx, a, next_task, ovf_list, ovf_n, task_list, d_ntask);
    else launch_xd16_r<4, C>(ctx, a, next_task, ovf_list, ovf_n, task_list, d_ntask);
}

static pastis_status align_qt(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets, int32_t n_q,
                              const uint8_t *d_tcodes, const int64_t *d_toffsets, int32_t n_t,
                              const pastis_cand *d_pairs, int64_t n_pairs, const pastis_params *params,
                              pastis_aln *d_out, int64_t *d_cells, const align_graph *g = nullptr) {
    if (!ctx || n_pairs < 0 || n_q < 0 || n_t < 0) return PASTIS_ERR_INVALID_ARG;
    pastis_status s = check_params(params);
    if (s != PASTIS_OK) return s;
    if (n_pairs == 0) return PASTIS_OK;
    if (!d_qcodes || !d_qoffsets || !d_tcodes || !d_toffsets || !d_pairs || !d_out || n_q == 0 || n_t == 0)
        return PASTIS_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    int8_t *dmat;
    PASTIS_WS(dmat, ctx, WS_FLAGS, 1024);
    int *flags = (int *)(dmat + 768);   // [0] error, [1] [3] [8] pair counters, [2] max length, [4] bad pair,
                                        // [5] bad code, [6..7] [12..13] [14..15] [16..17] task counters,
                                        // [9] [18] the 16-bit x-drop's deferred tasks (without, with carries)
    // the matrix, then the pass-1 layout at dmat + 640
    uint8_t hconst[640 + PASTIS_SW_BINS];
    memcpy(hconst, params->matrix, 576);
    memset(hconst + 576, 0, 64);
    memcpy(hconst + 640, ctx->sw_lay.extra, PASTIS_SW_BINS);
    if (!g) PASTIS_CUDA_TRY(cudaMemcpyAsync(dmat, hconst, sizeof(hconst), cudaMemcpyHostToDevice, st));
    PASTIS_CUDA_TRY(cudaMemsetAsync(flags, 0, 80, st));
    const int xd = params->mode == PASTIS_XD || params->mode == PASTIS_XD_FILTERED;
    const int xd_filtered = params->mode == PASTIS_XD_FILTERED;
    const int64_t *dn = g ? g->dc : nullptr;
    const int *chk = g ? flags + 4 : nullptr;
    if (g) {
        // the plan checked the lengths on the host; the pairs and the query residues here
        k_check_pairs<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(d_pairs, n_pairs, d_qoffsets, n_q,
                                                                         d_toffsets, n_t, params->k, xd, flags + 4,
                                                                         g->dc);
        PASTIS_LAUNCHED(ctx);
        const int blocks_c = (int)std::min<int64_t>(ceil_div64(g->qres_cap, 256), (int64_t)ctx->sm_count * 16);
        k_check_codes<<<blocks_c, 256, 0, st>>>(d_qcodes, g->qres_cap, flags + 5, g->dc + 1);
        PASTIS_LAUNCHED(ctx);
    }
    int lmax = g ? g->lmax : 0;
    if (!g) {
        k_max_len<<<(unsigned)ceil_div64(n_q, 256), 256, 0, st>>>(d_qoffsets, n_q, flags + 2);
        PASTIS_LAUNCHED(ctx);
        k_max_len<<<(unsigned)ceil_div64(n_t, 256), 256, 0, st>>>(d_toffsets, n_t, flags + 2);
        PASTIS_LAUNCHED(ctx);
        k_check_pairs<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(d_pairs, n_pairs, d_qoffsets, n_q,
                                                                         d_toffsets, n_t, params->k, xd, flags + 4,
                                                                         nullptr);
        PASTIS_LAUNCHED(ctx);
        int64_t h_end[2] = {0, 0};
        PASTIS_CUDA_TRY(cudaMemcpyAsync(&h_end[0], d_qoffsets + n_q, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PASTIS_CUDA_TRY(cudaMemcpyAsync(&h_end[1], d_toffsets + n_t, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int w = 0; w < 2; ++w) {
            const uint8_t *cd = w == 0 ? d_qcodes : d_tcodes;
            if (h_end[w] > 0 && (w == 0 || cd != d_qcodes)) {
                int blocks_c = (int)std::min<int64_t>(ceil_div64(h_end[w], 256), (int64_t)ctx->sm_count * 16);
                prof_begin(ctx, "align_checks");
                k_check_codes<<<blocks_c, 256, 0, st>>>(cd, h_end[w], flags + 5, nullptr);
                PASTIS_LAUNCHED(ctx);
                prof_end(ctx);
            }
        }
        int hf[6];
        PASTIS_CUDA_TRY(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
        PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
        if (hf[4]) return PASTIS_ERR_INVALID_ARG;
        if (hf[5]) return PASTIS_ERR_INVALID_RESIDUE;
        lmax = hf[2];
    }
    if (lmax > PASTIS_MAX_LEN) return PASTIS_ERR_INVALID_ARG;
    int xd_per_sm = 2, xd1_per_sm = 2;        // CTAs per SM with carries, and without (fewer registers)
    if (xd) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&xd_per_sm, k_xd_ext<true>, ALN_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&xd1_per_sm, k_xd_ext<false>, ALN_THREADS, 0);
        if (xd_per_sm < 1) xd_per_sm = 1;
        if (xd1_per_sm < xd_per_sm) xd1_per_sm = xd_per_sm;
    }
    const int blocks = ctx->sm_count * xd_per_sm, blocks1 = ctx->sm_count * xd1_per_sm;
    const int nwarps = (xd_filtered ? blocks1 : blocks) * ALN_WARPS;     // per-warp fallback buffers
    if (!xd) {
        s = sw_align(ctx, d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs, n_pairs, params, dmat, flags, lmax,
                     d_out, d_cells, dn, chk);
        if (s != PASTIS_OK) return s;
    } else {
        const int W = lmax + 2;
        int32_t *gbuf;
        PASTIS_WS(gbuf, ctx, WS_ALN_SCRATCH, sizeof(int32_t) * 18 * (size_t)W * nwarps);
        ext_out *ext;
        PASTIS_WS(ext, ctx, WS_ALN_PASS1, sizeof(ext_out) * 4 * (size_t)n_pairs);
        const int64_t n4 = 4 * n_pairs;
        uint32_t *need;
        PASTIS_WS(need, ctx, WS_ALN_ORDER, sizeof(uint32_t) * (3 * (size_t)n4 + 4));
        uint32_t *off = need + n4, *list = off + n4 + 1;
        const int per_warp = ctx->xd_per_warp;
        const bool lanes16 = per_warp && xd16_params_fit(params->gap_open, params->gap_extend, params->xdrop);
        int smax = -64;
        for (int x = 0; x < PASTIS_NSYM * PASTIS_NSYM; ++x) smax = std::max(smax, (int)params->matrix[x]);
        const xd16_args a16{d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs, n_pairs, params->k, dmat,
                            params->gap_open, params->gap_extend, params->xdrop, smax, ext, dn, chk};
        if (!xd_filtered) {
            // every extension with carries: in 16-bit lanes where it fits (the others
            // listed in list[flags[18]]), else in 32-bit lanes
            prof_begin(ctx, "xd_extend");
            if (lanes16) {
                launch_xd16<true>(ctx, per_warp, a16, flags + 16, list, (uint32_t *)(flags + 18), nullptr, nullptr);
                PASTIS_LAUNCHED(ctx);
            }
            k_xd_ext<true><<<blocks, ALN_THREADS, 0, st>>>(d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs,
                                                           n_pairs, params->k, dmat, params->gap_open,
                                                           params->gap_extend, params->xdrop, gbuf, W, flags + 6, ext,
                                                           lanes16 ? list : nullptr,
                                                           lanes16 ? (uint32_t *)(flags + 18) : nullptr, dn, chk);
            PASTIS_LAUNCHED(ctx);
            prof_end(ctx);
        } else {
            // phase 1: every extension's score, end and cells; then the carried
            // statistics only for the seeds whose spans pass the coverage test
            prof_begin(ctx, "xd_extend");
            if (lanes16) {
                // in 16-bit lanes, per_warp extensions per warp; the tasks it cannot hold
                // are listed (list[flags[9]]) and run in 32-bit lanes
                launch_xd16<false>(ctx, per_warp, a16, flags + 14, list, (uint32_t *)(flags + 9), nullptr, nullptr);
                PASTIS_LAUNCHED(ctx);
            }
            k_xd_ext<false><<<blocks1, ALN_THREADS, 0, st>>>(d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs,
                                                            n_pairs, params->k, dmat, params->gap_open,
                                                            params->gap_extend, params->xdrop, gbuf, W, flags + 6,
                                                            ext, lanes16 ? list : nullptr,
                                                            lanes16 ? (uint32_t *)(flags + 9) : nullptr, dn, chk);
            PASTIS_LAUNCHED(ctx);
            prof_end(ctx);
            k_xd_mark<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(d_qoffsets, d_toffsets, d_pairs, n_pairs,
                                                                          params->k, params->cov_min_pct, ext, need,
                                                                          dn, chk);
            PASTIS_LAUNCHED(ctx);
            s = exclusive_scan_u32(ctx, need, off, n4);
            if (s != PASTIS_OK) return s;
            k_xd_tasks<<<(unsigned)ceil_div64(n4, 256), 256, 0, st>>>(need, off, n4, list);
            PASTIS_LAUNCHED(ctx);
            prof_begin(ctx, "xd_carry");
            if (lanes16) {
                // the flagged tasks (list[0 .. list[n4]) in 16-bit lanes with carries; the
                // ones it cannot hold are listed in need[flags[18]], no longer needed
                launch_xd16<true>(ctx, per_warp, a16, flags + 16, need, (uint32_t *)(flags + 18), list, list + n4);
                PASTIS_LAUNCHED(ctx);
            }
            k_xd_ext<true><<<blocks, ALN_THREADS, 0, st>>>(d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs,
                                                           n_pairs, params->k, dmat, params->gap_open,
                                                           params->gap_extend, params->xdrop, gbuf, W, flags + 12,
                                                           ext, lanes16 ? need : list,
                                                           lanes16 ? (uint32_t *)(flags + 18) : list + n4, dn, chk);
            PASTIS_LAUNCHED(ctx);
            prof_end(ctx);
        }
        prof_begin(ctx, "xd_combine");
        k_xd_combine<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(
            d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs, n_pairs, params->k, dmat, params->ani_min_pct,
            params->cov_min_pct, xd_filtered, ext, d_out, (unsigned long long *)d_cells, dn, chk);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    if (g) return PASTIS_OK;                 // the plan reads the flags after its launch
    int herr = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&herr, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    return herr ? PASTIS_ERR_INTERNAL : PASTIS_OK;
}

extern "C" pastis_status pastis_align_pairs(pastis_ctx *ctx, const uint8_t *d_codes, const int64_t *d_offsets,
                                            int32_t n_seqs, const pastis_cand *d_pairs, int64_t n_pairs,
                                            const pastis_params *params, pastis_aln *d_out, int64_t *d_cells) {
    return align_qt(ctx, d_codes, d_offsets, n_seqs, d_codes, d_offsets, n_seqs, d_pairs, n_pairs, params, d_out,
                    d_cells);
}

extern "C" pastis_status pastis_align_pairs_qt(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets,
                                               int32_t n_q, const uint8_t *d_tcodes, const int64_t *d_toffsets,
                                               int32_t n_t, const pastis_cand *d_pairs, int64_t n_pairs,
                                               const pastis_params *params, pastis_aln *d_out, int64_t *d_cells) {
    return align_qt(ctx, d_qcodes, d_qoffsets, n_q, d_tcodes, d_toffsets, n_t, d_pairs, n_pairs, params, d_out,
                    d_cells);
}

extern "C" pastis_status pastis_sw_layout_set(pastis_ctx *ctx, const uint8_t *h_extra) {
    if (!ctx) return PASTIS_ERR_INVALID_ARG;
    sw_layout lay;
    for (int b = 0; b < PASTIS_SW_BINS; ++b) {
        const int v = h_extra ? h_extra[b] : 0;
        if (v > PASTIS_SW_MAX_EXTRA && v != PASTIS_SW_INT32) return PASTIS_ERR_INVALID_ARG;
        lay.extra[b] = (uint8_t)v;
    }
    ctx->sw_lay = lay;
    return PASTIS_OK;
}

extern "C" pastis_status pastis_xd_layout_set(pastis_ctx *ctx, int32_t per_warp) {
    if (!ctx || (per_warp != 0 && per_warp != 1 && per_warp != 2 && per_warp != 4)) return PASTIS_ERR_INVALID_ARG;
    ctx->xd_per_warp = per_warp;
    return PASTIS_OK;
}

extern "C" int32_t pastis_xd_layout_get(const pastis_ctx *ctx) { return ctx ? ctx->xd_per_warp : -1; }

extern "C" pastis_status pastis_sw_layout_get(const pastis_ctx *ctx, uint8_t *h_extra) {
    if (!ctx || !h_extra) return PASTIS_ERR_INVALID_ARG;
    for (int b = 0; b < PASTIS_SW_BINS; ++b) h_extra[b] = ctx->sw_lay.extra[b];
    return PASTIS_OK;
}

// The score-and-end alignment under each uniform layout (the extra stripes of pass 1,
// then 32-bit lanes for every pair), the per-bin cycles of each run summed over reps;
// per bin the fastest layout when it beats the default by 2% or more.
extern "C" pastis_status pastis_autotune_sw(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets,
                                            int32_t n_q, const uint8_t *d_tcodes, const int64_t *d_toffsets,
                                            int32_t n_t, const pastis_cand *d_pairs, int64_t n_pairs,
                                            const pastis_params *params, int32_t reps, uint8_t *h_extra,
                                            int64_t *h_cycles) {
    if (!ctx || !params || reps < 1 || n_pairs < 0) return PASTIS_ERR_INVALID_ARG;
    pastis_status s = check_params(params);
    if (s != PASTIS_OK) return s;
    if (params->mode != PASTIS_SW && params->mode != PASTIS_SW_SCORE && params->mode != PASTIS_SW_FILTERED)
        return PASTIS_ERR_UNSUPPORTED;
    constexpr int NX = PASTIS_SW_MAX_EXTRA + 2;               // 0..MAX_EXTRA, then PASTIS_SW_INT32
    const sw_layout saved = ctx->sw_lay;
    int64_t cyc[NX * PASTIS_SW_BINS] = {0};
    if (n_pairs > 0) {
        unsigned long long *d_tune;
        PASTIS_WS(d_tune, ctx, WS_TUNE, sizeof(unsigned long long) * NX * PASTIS_SW_BINS +
                                            sizeof(pastis_aln) * (size_t)n_pairs + 16);
        pastis_aln *d_out = (pastis_aln *)(d_tune + NX * PASTIS_SW_BINS);
        PASTIS_CUDA_TRY(cudaMemsetAsync(d_tune, 0, sizeof(unsigned long long) * NX * PASTIS_SW_BINS, ctx->stream));
        pastis_params ps = *params;
        ps.mode = PASTIS_SW_SCORE;
        for (int r = 0; r < reps && s == PASTIS_OK; ++r) {
            for (int x = 0; x < NX && s == PASTIS_OK; ++x) {
                const uint8_t v = x <= PASTIS_SW_MAX_EXTRA ? (uint8_t)x : (uint8_t)PASTIS_SW_INT32;
                for (int b = 0; b < PASTIS_SW_BINS; ++b) ctx->sw_lay.extra[b] = v;
                ctx->d_tune = d_tune + x * PASTIS_SW_BINS;
                s = align_qt(ctx, d_qcodes, d_qoffsets, n_q, d_tcodes, d_toffsets, n_t, d_pairs, n_pairs, &ps, d_out,
                             nullptr);
            }
        }
        ctx->d_tune = nullptr;
        ctx->sw_lay = saved;
        if (s != PASTIS_OK) return s;
        PASTIS_CUDA_TRY(cudaMemcpyAsync(cyc, d_tune, sizeof(cyc), cudaMemcpyDeviceToHost, ctx->stream));
        PASTIS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    sw_layout best;
    for (int b = 0; b < PASTIS_SW_BINS; ++b) {
        int bx = 0;
        for (int x = 1; x < NX; ++x)
            if (cyc[x * PASTIS_SW_BINS + b] > 0 && cyc[x * PASTIS_SW_BINS + b] < cyc[bx * PASTIS_SW_BINS + b])
                bx = x;
        // keep the default unless the winner is clearly faster
        if (bx != 0 && (double)cyc[bx * PASTIS_SW_BINS + b] > 0.98 * (double)cyc[b]) bx = 0;
        best.extra[b] = bx <= PASTIS_SW_MAX_EXTRA ? (uint8_t)bx : (uint8_t)PASTIS_SW_INT32;
    }
    ctx->sw_lay = best;
    if (h_extra)
        for (int b = 0; b < PASTIS_SW_BINS; ++b) h_extra[b] = best.extra[b];
    if (h_cycles)
        for (int x = 0; x < NX * PASTIS_SW_BINS; ++x) h_cycles[x] = cyc[x];
    return PASTIS_OK;
}

// The x-drop lane layout: the filter-only x-drop of the pairs under each setting (32-bit
// lanes, then 1, 2 and 4 extensions per warp in 16-bit lanes), each call timed by CUDA
// events on the context's stream, the best of `reps`; the fastest setting when it beats
// the current one by 2% or more, else the current one.
extern "C" pastis_status pastis_autotune_xd(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets,
                                            int32_t n_q, const uint8_t *d_tcodes, const int64_t *d_toffsets,
                                            int32_t n_t, const pastis_cand *d_pairs, int64_t n_pairs,
                                            const pastis_params *params, int32_t reps, int32_t *h_per_warp,
                                            double *h_ms) {
    if (!ctx || !params || reps < 1 || n_pairs < 0) return PASTIS_ERR_INVALID_ARG;
    pastis_status s = check_params(params);
    if (s != PASTIS_OK) return s;
    if (params->mode != PASTIS_XD && params->mode != PASTIS_XD_FILTERED) return PASTIS_ERR_UNSUPPORTED;
    constexpr int NX = 4;
    const int choice[NX] = {0, 1, 2, 4};
    const int saved = ctx->xd_per_warp;
    double ms[NX] = {0.0, 0.0, 0.0, 0.0};
    if (n_pairs > 0) {
        pastis_aln *d_out;
        PASTIS_WS(d_out, ctx, WS_TUNE, sizeof(pastis_aln) * (size_t)n_pairs + 16);
        const pastis_params &ps = *params;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
            cudaGetLastError();
            if (ev[0]) cudaEventDestroy(ev[0]);
            return PASTIS_ERR_CUDA;
        }
        for (int r = 0; r < reps && s == PASTIS_OK; ++r) {
            for (int x = 0; x < NX && s == PASTIS_OK; ++x) {
                ctx->xd_per_warp = choice[x];
                if (cudaEventRecord(ev[0], ctx->stream) != cudaSuccess) { s = PASTIS_ERR_CUDA; break; }
                s = align_qt(ctx, d_qcodes, d_qoffsets, n_q, d_tcodes, d_toffsets, n_t, d_pairs, n_pairs, &ps, d_out,
                             nullptr);
                float t = 0.f;
                if (s == PASTIS_OK && (cudaEventRecord(ev[1], ctx->stream) != cudaSuccess ||
                                       cudaEventSynchronize(ev[1]) != cudaSuccess ||
                                       cudaEventElapsedTime(&t, ev[0], ev[1]) != cudaSuccess))
                    s = PASTIS_ERR_CUDA;
                if (s == PASTIS_OK && (r == 0 || t < ms[x])) ms[x] = t;
            }
        }
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        ctx->xd_per_warp = saved;
        if (s != PASTIS_OK) { cudaGetLastError(); return s; }
        int cur = 0, bx = 0;
        for (int x = 0; x < NX; ++x) {
            if (choice[x] == saved) cur = x;
            if (ms[x] < ms[bx]) bx = x;
        }
        if (ms[bx] > 0.98 * ms[cur]) bx = cur;
        ctx->xd_per_warp = choice[bx];
    }
    if (h_per_warp) *h_per_warp = ctx->xd_per_warp;
    if (h_ms)
        for (int x = 0; x < NX; ++x) h_ms[x] = ms[x];
    return PASTIS_OK;
}

// ---------------------------------------------------------------------------------
// Alignment plans: the whole alignment of one batch captured once as a CUDA graph over
// fixed-capacity buffers, replayed per batch with the counts in device memory.
// ---------------------------------------------------------------------------------
struct pastis_align_plan {
    pastis_ctx *ctx;                 // private workspace on the plan's own stream
    cudaStream_t stream;             // non-blocking: capture is not possible on a default stream
    cudaStream_t caller;             // the stream of the context the plan was made from
    cudaEvent_t ready;               // orders each run after the caller's earlier work
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    uint8_t *qcodes;
    int64_t *qoffsets;
    pastis_cand *pairs;
    pastis_aln *out;
    int64_t *dc;                     // [0] pairs, [1] query residues, [2] queries
    int64_t *h_dc;                   // pinned staging of dc
    const uint8_t *tcodes;
    const int64_t *toffsets;
    int32_t n_t, max_q, max_len;
    int64_t max_qres, max_pairs;
    pastis_params params;
};

static void plan_free(pastis_align_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->qcodes) cudaFree(p->qcodes);
    if (p->qoffsets) cudaFree(p->qoffsets);
    if (p->pairs) cudaFree(p->pairs);
    if (p->out) cudaFree(p->out);
    if (p->dc) cudaFree(p->dc);
    if (p->h_dc) cudaFreeHost(p->h_dc);
    if (p->ctx) pastis_ctx_destroy(p->ctx);
    if (p->ready) cudaEventDestroy(p->ready);
    if (p->stream) cudaStreamDestroy(p->stream);
    free(p);
}

extern "C" pastis_status pastis_align_plan_create(pastis_ctx *ctx, const uint8_t *d_tcodes, const int64_t *d_toffsets,
                                                  int32_t n_t, int32_t max_q, int64_t max_qres, int64_t max_pairs,
                                                  int32_t max_len, const pastis_params *params,
                                                  pastis_align_plan **out) {
    if (!out) return PASTIS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ctx || !d_tcodes || !d_toffsets || n_t < 1 || max_q < 1 || max_qres < 1 || max_pairs < 1 || max_len < 1 ||
        max_len > PASTIS_MAX_LEN || max_q > INT32_MAX - 1)
        return PASTIS_ERR_INVALID_ARG;
    pastis_status s = check_params(params);
    if (s != PASTIS_OK) return s;
    cudaStream_t st = ctx->stream;
    // the targets once: lengths within max_len, codes valid
    int *tf;
    PASTIS_WS(tf, ctx, WS_FLAGS, 1024);
    int *fl = (int *)((int8_t *)tf + 768);
    PASTIS_CUDA_TRY(cudaMemsetAsync(fl, 0, 64, st));
    k_max_len<<<(unsigned)ceil_div64(n_t, 256), 256, 0, st>>>(d_toffsets, n_t, fl + 2);
    PASTIS_LAUNCHED(ctx);
    int64_t t_end = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&t_end, d_toffsets + n_t, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    if (t_end > 0) {
        const int blocks_c = (int)std::min<int64_t>(ceil_div64(t_end, 256), (int64_t)ctx->sm_count * 16);
        k_check_codes<<<blocks_c, 256, 0, st>>>(d_tcodes, t_end, fl + 5, nullptr);
        PASTIS_LAUNCHED(ctx);
    }
    int hf[6];
    PASTIS_CUDA_TRY(cudaMemcpyAsync(hf, fl, sizeof(hf), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hf[5]) return PASTIS_ERR_INVALID_RESIDUE;
    if (hf[2] > max_len) return PASTIS_ERR_INVALID_ARG;

    pastis_align_plan *p = (pastis_align_plan *)calloc(1, sizeof(pastis_align_plan));
    if (!p) return PASTIS_ERR_OUT_OF_MEMORY;
    p->tcodes = d_tcodes; p->toffsets = d_toffsets; p->n_t = n_t;
    p->max_q = max_q; p->max_qres = max_qres; p->max_pairs = max_pairs; p->max_len = max_len;
    p->params = *params;
    p->caller = st;
    if (cudaSetDevice(ctx->device) != cudaSuccess || cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ready, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        plan_free(p);
        return PASTIS_ERR_CUDA;
    }
    st = p->stream;
    s = pastis_ctx_create(&p->ctx, ctx->device, (void *)st);
    if (s != PASTIS_OK) { plan_free(p); return s; }
    p->ctx->sw_lay = ctx->sw_lay;
    p->ctx->xd_per_warp = ctx->xd_per_warp;
#define PLAN_TRY(expr) do { if ((expr) != cudaSuccess) { cudaGetLastError(); plan_free(p); return PASTIS_ERR_OUT_OF_MEMORY; } } while (0)
    PLAN_TRY(cudaMalloc(&p->qcodes, (size_t)max_qres + 16));
    PLAN_TRY(cudaMalloc(&p->qoffsets, sizeof(int64_t) * ((size_t)max_q + 1)));
    PLAN_TRY(cudaMalloc(&p->pairs, sizeof(pastis_cand) * (size_t)max_pairs));
    PLAN_TRY(cudaMalloc(&p->out, sizeof(pastis_aln) * (size_t)max_pairs));
    PLAN_TRY(cudaMalloc(&p->dc, sizeof(int64_t) * 4));
    PLAN_TRY(cudaMallocHost(&p->h_dc, sizeof(int64_t) * 4));
#undef PLAN_TRY
    s = PASTIS_ERR_CUDA;
    do {
        if (cudaMemsetAsync(p->qcodes, 0, (size_t)max_qres + 16, st) != cudaSuccess) break;
        if (cudaMemsetAsync(p->qoffsets, 0, sizeof(int64_t) * ((size_t)max_q + 1), st) != cudaSuccess) break;
        if (cudaMemsetAsync(p->dc, 0, sizeof(int64_t) * 4, st) != cudaSuccess) break;
        // the private context's constants: the matrix and the pass-1 layout
        int8_t *dmat = (int8_t *)ws_get(p->ctx, WS_FLAGS, 1024);
        if (!dmat) { s = PASTIS_ERR_OUT_OF_MEMORY; break; }
        uint8_t hconst[640 + PASTIS_SW_BINS];
        memcpy(hconst, params->matrix, 576);
        memset(hconst + 576, 0, 64);
        memcpy(hconst + 640, p->ctx->sw_lay.extra, PASTIS_SW_BINS);
        if (cudaMemcpyAsync(dmat, hconst, sizeof(hconst), cudaMemcpyHostToDevice, st) != cudaSuccess) break;
        align_graph g{p->dc, max_len, max_qres};
        // a run with every count 0 sizes the workspace, so the capture allocates nothing
        s = align_qt(p->ctx, p->qcodes, p->qoffsets, max_q, d_tcodes, d_toffsets, n_t, p->pairs, max_pairs,
                     &p->params, p->out, nullptr, &g);
        if (s != PASTIS_OK) break;
        s = PASTIS_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) break;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) break;
        const int64_t launches = p->ctx->launches;
        pastis_status cs = align_qt(p->ctx, p->qcodes, p->qoffsets, max_q, d_tcodes, d_toffsets, n_t, p->pairs,
                                    max_pairs, &p->params, p->out, nullptr, &g);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(st, &graph);
        p->graph = graph;
        p->ctx->launches = launches;     // counted per replay instead
        if (cs != PASTIS_OK) { s = cs; break; }
        if (ce != cudaSuccess || !graph) break;
        if (cudaGraphInstantiate(&p->exec, graph, 0) != cudaSuccess) break;
        s = PASTIS_OK;
    } while (0);
    if (s != PASTIS_OK) {
        cudaGetLastError();
        plan_free(p);
        return s;
    }
    *out = p;
    return PASTIS_OK;
}

extern "C" pastis_status pastis_align_plan_run(pastis_align_plan *p, const uint8_t *d_qcodes,
                                               const int64_t *h_qoffsets, int32_t n_q, const pastis_cand *d_pairs,
                                               int64_t n_pairs, pastis_aln *d_out) {
    if (!p || !h_qoffsets || n_q < 1 || n_pairs < 0) return PASTIS_ERR_INVALID_ARG;
    if (h_qoffsets[0] != 0) return PASTIS_ERR_INVALID_ARG;
    for (int32_t q = 0; q < n_q; ++q)
        if (h_qoffsets[q + 1] < h_qoffsets[q]) return PASTIS_ERR_INVALID_ARG;
    if (n_q > p->max_q || n_pairs > p->max_pairs || h_qoffsets[n_q] > p->max_qres) return PASTIS_ERR_CAPACITY;
    for (int32_t q = 0; q < n_q; ++q)
        if (h_qoffsets[q + 1] - h_qoffsets[q] > p->max_len) return PASTIS_ERR_CAPACITY;
    if (n_pairs == 0) return PASTIS_OK;
    if (!d_pairs || !d_out || (h_qoffsets[n_q] > 0 && !d_qcodes)) return PASTIS_ERR_INVALID_ARG;
    cudaStream_t st = p->stream;
    PASTIS_CUDA_TRY(cudaEventRecord(p->ready, p->caller));      // the batch was made on the caller's stream
    PASTIS_CUDA_TRY(cudaStreamWaitEvent(st, p->ready, 0));
    PASTIS_CUDA_TRY(cudaMemcpyAsync(p->qoffsets, h_qoffsets, sizeof(int64_t) * ((size_t)n_q + 1),
                                    cudaMemcpyHostToDevice, st));
    if (h_qoffsets[n_q] > 0)
        PASTIS_CUDA_TRY(cudaMemcpyAsync(p->qcodes, d_qcodes, (size_t)h_qoffsets[n_q], cudaMemcpyDeviceToDevice, st));
    PASTIS_CUDA_TRY(cudaMemcpyAsync(p->pairs, d_pairs, sizeof(pastis_cand) * (size_t)n_pairs,
                                    cudaMemcpyDeviceToDevice, st));
    p->h_dc[0] = n_pairs;
    p->h_dc[1] = h_qoffsets[n_q];
    p->h_dc[2] = n_q;
    p->h_dc[3] = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(p->dc, p->h_dc, sizeof(int64_t) * 4, cudaMemcpyHostToDevice, st));
    PASTIS_CUDA_TRY(cudaGraphLaunch(p->exec, st));
    p->ctx->launches++;
    int hf[6];
    const int *fl = (const int *)((const int8_t *)p->ctx->ws[WS_FLAGS] + 768);
    PASTIS_CUDA_TRY(cudaMemcpyAsync(hf, fl, sizeof(hf), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hf[4]) return PASTIS_ERR_INVALID_ARG;
    if (hf[5]) return PASTIS_ERR_INVALID_RESIDUE;
    if (hf[0]) return PASTIS_ERR_INTERNAL;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(d_out, p->out, sizeof(pastis_aln) * (size_t)n_pairs, cudaMemcpyDeviceToDevice, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    return PASTIS_OK;
}

extern "C" pastis_status pastis_align_plan_destroy(pastis_align_plan *p) {
    if (!p) return PASTIS_ERR_INVALID_ARG;
    if (p->stream) cudaStreamSynchronize(p->stream);
    plan_free(p);
    return PASTIS_OK;
}

extern "C" int64_t pastis_align_plan_graph_nodes(const pastis_align_plan *p) {
    size_t n = 0;
    if (!p || !p->graph || cudaGraphGetNodes(p->graph, nullptr, &n) != cudaSuccess) return -1;
    return (int64_t)n;
}
