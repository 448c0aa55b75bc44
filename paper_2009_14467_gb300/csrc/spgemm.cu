// a6-a7: candidate discovery, B = A A^T or (A S) A^T, with symmetrization.
//
// Sec. IV-A: the multiply of the semiring pairs the start positions of a shared k-mer,
// the add counts shared k-mers and keeps at most two seeds (here: the two shared
// k-mers of smallest code); B is symmetric, so only i < j is formed.  Sec. IV-C: with
// substitutes the left operand is AS.  Symmetrization (a separate component in the
// paper's dissection, Sec. VI-A) is fused: the row of i is formed in both orientations,
// (AS)_i . A_j and A_i . (AS)_j, and each pair keeps the orientation that shares more
// (i -> j on ties).
//
// Row-wise hash SpGEMM in two kernels.
//  * Cursors: one warp per row i.  Each left entry t of the row (a k-mer of AS_i, and of
//    A_i for the second orientation) finds where its posting list (sorted by sequence)
//    reaches the row's first column j >= jlo; entries with a non-empty rest keep a
//    cursor (next j, posting index, posting end).  The warp also sums the row's exact
//    product count.
//  * Rows: one CTA per row, a hash table in shared memory keyed by j (count and two
//    seeds per orientation).  A row whose products could overflow the table is formed
//    in column ranges [a, z), in order; each range advances every cursor up to z, so
//    each posting entry is visited once however many ranges the row takes.  An entry
//    inserts count += 1 and the seed t << 16 | pos_j into a two-smallest pair with
//        old = atomicMin(s0, v);  atomicMin(s1, max(old, v))
//    which leaves s0, s1 = the two smallest values whatever the arrival order.  Row
//    entries are in ascending code order, so the smallest t is the smallest code.  After
//    each range the CTA compacts the entries that pass min_shared, sorts them by j
//    (bitonic) and appends their records to the row's slice; a table that overflows
//    (more distinct j than it holds) resets the cursors to the range start and halves
//    the range.  A final pass concatenates the slices in row order.
#include <algorithm>
#include <vector>

#include "internal.cuh"

pastis_status build_as(pastis_ctx *ctx, const pastis_kmat *A, const pastis_params *p, as_matrix *out);

namespace {

constexpr int SPG_THREADS = 256;
constexpr int SPG_THREADS_MAX = 1024;
// Threads of a row CTA: the largest tables leave room for one or two CTAs per SM, so
// their CTAs are wider, keeping up to 32 warps per SM on the posting-list gathers.
static int spg_threads_for(int tsize) { return tsize >= 4096 ? 1024 : (tsize >= 2048 ? 512 : SPG_THREADS); }
constexpr int CUR_THREADS = 256;
constexpr uint64_t SEED_NONE = ~0ull;
constexpr int32_t J_DONE = 0x7FFFFFFF;     // cursor past its posting list
constexpr uint32_t SIDE_B = 0x80000000u;   // cursor of the second orientation

struct operand {          // one side of the product: left rows and right posting lists
    const int64_t *row_ptr;
    const uint32_t *row_code;
    const uint16_t *row_pos;
    const uint32_t *col_ptr;
    const int32_t *col_seq;
    const uint16_t *col_pos;
};

struct cursors {          // per kept left entry of the rows of one call
    int32_t *nj;          // next column j of the entry (J_DONE when exhausted)
    uint32_t *t;          // entry index within its row | SIDE_B
    int64_t *x;           // posting index of nj
    int64_t *pe;          // end of the posting list
};

struct row_item {
    int32_t i;
    int32_t pieces;       // column ranges the row starts with
    int64_t ent_off;      // first cursor of the row
    int64_t n_act;        // cursors of the row
    int64_t out_off;      // slice in the temporary record buffer
    int64_t out_cap;
};

__device__ __forceinline__ uint32_t hash_j(int32_t j) { return (uint32_t)j * 2654435761u; }

__device__ __forceinline__ int64_t lower_bound_seq(const int32_t *seq, int64_t a, int64_t b, int32_t key) {
    // first index in [a, b) with seq >= key
    if (b - a <= 8) {
        while (a < b && seq[a] < key) ++a;
        return a;
    }
    while (a < b) {
        int64_t mid = (a + b) >> 1;
        if (seq[mid] < key) a = mid + 1; else b = mid;
    }
    return a;
}

// Cursors of the rows rows[w] (one warp each): entries with postings at j >= jlo, in
// entry order (first orientation, then the second), their count and the row's products.
__global__ void __launch_bounds__(CUR_THREADS) k_spgemm_cursors(operand F, operand B, int subs, int self,
                                                               const int32_t *rows, const int64_t *ent_off,
                                                               int32_t n_rows, cursors cur, int64_t *n_act,
                                                               int64_t *n_prod, unsigned long long *stats) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_rows) return;
    const int32_t i = rows[w];
    const int32_t jlo = self ? i + 1 : 0;
    const int64_t base = ent_off[w];
    int64_t cnt = 0, prod = 0, left = 0;
    for (int side = 0; side <= subs; ++side) {
        const operand &L = side ? B : F;
        const int64_t rb = L.row_ptr[i], re = L.row_ptr[i + 1];
        left += re - rb;
        for (int64_t t0 = rb; t0 < re; t0 += 32) {
            const int64_t t = t0 + lane;
            bool act = false;
            int64_t x = 0, pe = 0;
            int32_t nj = 0;
            if (t < re) {
                const uint32_t c = L.row_code[t];
                const int64_t pb = L.col_ptr[c];
                pe = L.col_ptr[c + 1];
                if (pe > pb) {
                    x = lower_bound_seq(L.col_seq, pb, pe, jlo);
                    if (x < pe) { act = true; nj = L.col_seq[x]; }
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, act);
            if (act) {
                const int64_t pos = base + cnt + __popc(m & ((1u << lane) - 1u));
                cur.nj[pos] = nj;
                cur.t[pos] = (uint32_t)(t - rb) | (side ? SIDE_B : 0u);
                cur.x[pos] = x;
                cur.pe[pos] = pe;
                prod += pe - x;
            }
            cnt += __popc(m);
        }
    }
    for (int d = 16; d > 0; d >>= 1) prod += __shfl_down_sync(0xffffffffu, prod, d);
    if (lane == 0) {
        n_act[w] = cnt;
        n_prod[w] = prod;
        if (stats) {
            atomicAdd(&stats[0], (unsigned long long)prod);
            atomicAdd(&stats[1], (unsigned long long)left);
        }
    }
}

__device__ void bitonic_sort_pairs(uint32_t *key, uint32_t *val, int n) {
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int x = threadIdx.x; x < n / 2; x += blockDim.x) {
                int lo = 2 * x - (x & (stride - 1));
                int hi = lo + stride;
                bool up = ((lo & size) == 0);
                uint32_t a = key[lo], b = key[hi];
                if ((a > b) == up) {
                    key[lo] = b; key[hi] = a;
                    uint32_t t = val[lo]; val[lo] = val[hi]; val[hi] = t;
                }
            }
            __syncthreads();
        }
    }
}

// Exclusive prefix sums of the popcounts of bits[0, nw) into pre[0, nw), by the whole
// CTA; returns the total.  Each thread takes a contiguous run of words.
__device__ uint32_t block_popc_scan(const uint32_t *bits, uint32_t *pre, int nw, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int per = (nw + (int)blockDim.x - 1) / (int)blockDim.x;
    const int w0 = min(nw, (int)threadIdx.x * per), w1 = min(nw, w0 + per);
    uint32_t sum = 0;
    for (int w = w0; w < w1; ++w) sum += __popc(bits[w]);
    uint32_t incl = sum;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t off = 0, total = 0;
    for (int q = 0; q < nwarp; ++q) {
        const uint32_t v = s_warp[q];
        off += q < warp ? v : 0u;
        total += v;
    }
    uint32_t run = off + incl - sum;
    for (int w = w0; w < w1; ++w) {
        pre[w] = run;
        run += __popc(bits[w]);
    }
    __syncthreads();
    return total;
}

// One CTA per row (items of one table size).  SUBS: two orientations per entry
// (fwd = (AS)_i A_j, bwd = A_i (AS)_j).  Shared memory: s0[T], s1[T] (+ b0[T], b1[T]),
// key[T], cnt[T] (+ cnt_b[T]), then scratch key[T], val[T].
// The passing entries of a range [a, z) leave in column order.  When the range is at
// most 32 T columns wide (the scratch holds a bitmap of it and the popcount prefix of
// its words), each passing column sets its bit, and an entry's place is the number of
// set bits before it: no sort.  Otherwise the entries are compacted and bitonic-sorted.
// The bitmap path clears each slot as it writes it, so the next range starts on a clean
// table; the sort path clears the whole table at the start of the next range.
template <bool SUBS>
__global__ void __launch_bounds__(SPG_THREADS_MAX) k_spgemm_rows(operand F, operand B, const row_item *items,
                                                             int tsize, int32_t min_shared, int self, int32_t n_cols,
                                                             cursors cur, pastis_cand *tmp_out, int64_t *item_count,
                                                             int *item_error, unsigned long long *stats) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *s_s0 = (unsigned long long *)smem;
    unsigned long long *s_s1 = s_s0 + tsize;
    unsigned long long *s_b0 = s_s1 + tsize;                      // SUBS only
    unsigned long long *s_b1 = SUBS ? s_b0 + tsize : s_b0;
    int32_t *s_key = (int32_t *)(SUBS ? s_b1 + tsize : s_s1 + tsize);
    uint32_t *s_cnt = (uint32_t *)(s_key + tsize);
    uint32_t *s_cntb = s_cnt + tsize;                             // SUBS only
    uint32_t *s_sk = SUBS ? s_cntb + tsize : s_cnt + tsize;
    uint32_t *s_sv = s_sk + tsize;
    __shared__ int s_overflow;
    __shared__ int s_nvalid;

    const row_item it = items[blockIdx.x];
    const int32_t i = it.i;
    const int32_t jlo = self ? i + 1 : 0;
    const int64_t e0 = it.ent_off, ne = it.n_act;
    const int64_t rb_f = F.row_ptr[i];
    const int64_t rb_b = SUBS ? B.row_ptr[i] : 0;
    int64_t width = ((int64_t)n_cols - jlo + it.pieces - 1) / it.pieces;
    int64_t out_n = 0;
    unsigned long long n_rec = 0;
    __shared__ uint32_t s_warp[SPG_THREADS_MAX / 32];
    int64_t a = jlo;
    int guard = 0;
    bool dirty = true;                           // the table holds entries of an earlier range
    while (a < n_cols) {
        const int32_t z = (int32_t)(a + width < (int64_t)n_cols ? a + width : (int64_t)n_cols);
        if (dirty) {
            for (int x = threadIdx.x; x < tsize; x += blockDim.x) {
                s_key[x] = -1;
                s_cnt[x] = 0;
                s_s0[x] = SEED_NONE;
                s_s1[x] = SEED_NONE;
                if (SUBS) { s_cntb[x] = 0; s_b0[x] = SEED_NONE; s_b1[x] = SEED_NONE; }
            }
        }
        dirty = true;
        if (threadIdx.x == 0) { s_overflow = 0; s_nvalid = 0; }
        __syncthreads();
        // every cursor up to z
        volatile int *ovf = &s_overflow;
        for (int64_t e = e0 + threadIdx.x; e < e0 + ne; e += blockDim.x) {
            if (*ovf) break;                     // the range is redone anyway
            int32_t j = cur.nj[e];
            if (j >= z) continue;
            const uint32_t tt = cur.t[e];
            const bool sb = SUBS && (tt & SIDE_B);
            const int32_t *cs = sb ? B.col_seq : F.col_seq;
            const uint16_t *cp = sb ? B.col_pos : F.col_pos;
            uint32_t *cnt = sb ? s_cntb : s_cnt;
            unsigned long long *q0 = sb ? s_b0 : s_s0, *q1 = sb ? s_b1 : s_s1;
            const unsigned long long tv = (unsigned long long)(tt & ~SIDE_B) << 16;
            int64_t x = cur.x[e];
            const int64_t pe = cur.pe[e];
            bool full = false;
            for (;;) {
                uint32_t slot = hash_j(j) & (uint32_t)(tsize - 1);
                int probes = 0;
                for (;;) {
                    const int32_t prev = atomicCAS(&s_key[slot], -1, j);
                    if (prev == -1 || prev == j) break;
                    slot = (slot + 1) & (uint32_t)(tsize - 1);
                    if (++probes >= tsize) { full = true; break; }
                }
                if (full) break;
                atomicAdd(&cnt[slot], 1u);
                const unsigned long long v = tv | (unsigned long long)cp[x];
                const unsigned long long old = atomicMin(&q0[slot], v);
                atomicMin(&q1[slot], old > v ? old : v);
                if (++x >= pe) { j = J_DONE; break; }
                j = cs[x];
                if (j >= z) break;
            }
            if (full) { s_overflow = 1; continue; }
            cur.x[e] = x;
            cur.nj[e] = j;
        }
        __syncthreads();
        if (s_overflow) {
            // more distinct j in [a, z) than the table holds: every cursor back to a,
            // and the range halved
            for (int64_t e = e0 + threadIdx.x; e < e0 + ne; e += blockDim.x) {
                const uint32_t tt = cur.t[e];
                const bool sb = SUBS && (tt & SIDE_B);
                const operand &L = sb ? B : F;
                const int64_t t = (sb ? rb_b : rb_f) + (int64_t)(tt & ~SIDE_B);
                const int64_t pb = L.col_ptr[L.row_code[t]], pe = cur.pe[e];
                const int64_t x = lower_bound_seq(L.col_seq, pb, pe, (int32_t)a);
                cur.x[e] = x;
                cur.nj[e] = x < pe ? L.col_seq[x] : J_DONE;
            }
            __syncthreads();
            if (z - a <= 1 || ++guard > 64) {          // cannot happen: one column fits any table
                if (threadIdx.x == 0) { item_error[blockIdx.x] = 1; item_count[blockIdx.x] = 0; }
                return;
            }
            width = (z - a) / 2;
            continue;
        }
        const int64_t wid = (int64_t)z - a;
        if (wid <= (int64_t)tsize * 32) {
            // the bitmap of the passing columns of [a, z), then each entry's rank
            uint32_t *bits = s_sk, *pre = s_sv;
            const int nw = (int)((wid + 31) >> 5);
            for (int x = threadIdx.x; x < nw; x += blockDim.x) bits[x] = 0u;
            __syncthreads();
            for (int x = threadIdx.x; x < tsize; x += blockDim.x) {
                const int32_t j = s_key[x];
                if (j < 0) continue;
                uint32_t c = s_cnt[x];
                if (SUBS && s_cntb[x] > c) c = s_cntb[x];
                if ((int64_t)c < (int64_t)min_shared) continue;
                const uint32_t off = (uint32_t)(j - (int32_t)a);
                atomicOr(&bits[off >> 5], 1u << (off & 31));
            }
            __syncthreads();
            const int nv = (int)block_popc_scan(bits, pre, nw, s_warp);
            if (out_n + nv > it.out_cap) {   // cannot happen: the capacity is the row's products
                if (threadIdx.x == 0) { item_error[blockIdx.x] = 1; item_count[blockIdx.x] = 0; }
                return;
            }
            for (int x = threadIdx.x; x < tsize; x += blockDim.x) {
                const int32_t j = s_key[x];
                if (j < 0) continue;
                const uint32_t off = (uint32_t)(j - (int32_t)a);
                const uint32_t word = bits[off >> 5], bit = 1u << (off & 31);
                if (word & bit) {
                    pastis_cand rec;
                    rec.i = i;
                    rec.j = j;
                    const bool use_b = SUBS && (s_cntb[x] > s_cnt[x]);
                    unsigned long long sd[2];
                    int64_t rb;
                    const uint16_t *lpos;
                    if (use_b) {
                        rec.count = s_cntb[x]; sd[0] = s_b0[x]; sd[1] = s_b1[x]; rb = rb_b; lpos = B.row_pos;
                    } else {
                        rec.count = s_cnt[x]; sd[0] = s_s0[x]; sd[1] = s_s1[x]; rb = rb_f; lpos = F.row_pos;
                    }
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        if (sd[q] == SEED_NONE) { rec.qpos[q] = 0xFFFF; rec.tpos[q] = 0xFFFF; continue; }
                        const int64_t t = (int64_t)(sd[q] >> 16);
                        rec.qpos[q] = lpos[rb + t];
                        rec.tpos[q] = (uint16_t)(sd[q] & 0xFFFF);
                    }
                    const int r = (int)pre[off >> 5] + __popc(word & (bit - 1u));
                    tmp_out[it.out_off + out_n + r] = rec;
                }
                // clear the slot for the next range
                s_key[x] = -1;
                s_cnt[x] = 0;
                s_s0[x] = SEED_NONE;
                s_s1[x] = SEED_NONE;
                if (SUBS) { s_cntb[x] = 0; s_b0[x] = SEED_NONE; s_b1[x] = SEED_NONE; }
            }
            out_n += nv;
            n_rec += (unsigned long long)nv;
            dirty = false;
            __syncthreads();
            a = z;
            continue;
        }
        // compact the passing entries of [a, z), sort them by j, append their records
        for (int x = threadIdx.x; x < tsize; x += blockDim.x) {
            if (s_key[x] < 0) continue;
            uint32_t c = s_cnt[x];
            if (SUBS && s_cntb[x] > c) c = s_cntb[x];
            if ((int64_t)c < (int64_t)min_shared) continue;
            const int r = atomicAdd(&s_nvalid, 1);
            s_sk[r] = (uint32_t)s_key[x];
            s_sv[r] = (uint32_t)x;
        }
        __syncthreads();
        const int nv = s_nvalid;
        int np2 = 1;
        while (np2 < nv) np2 <<= 1;
        for (int x = nv + threadIdx.x; x < np2; x += blockDim.x) { s_sk[x] = 0xFFFFFFFFu; s_sv[x] = 0; }
        __syncthreads();
        bitonic_sort_pairs(s_sk, s_sv, np2);
        if (out_n + nv > it.out_cap) {   // cannot happen: the capacity is the row's products
            if (threadIdx.x == 0) { item_error[blockIdx.x] = 1; item_count[blockIdx.x] = 0; }
            return;
        }
        for (int r = threadIdx.x; r < nv; r += blockDim.x) {
            const int slot = (int)s_sv[r];
            pastis_cand rec;
            rec.i = i;
            rec.j = (int32_t)s_sk[r];
            const bool use_b = SUBS && (s_cntb[slot] > s_cnt[slot]);
            unsigned long long sd[2];
            int64_t rb;
            const uint16_t *lpos;
            if (use_b) {
                rec.count = s_cntb[slot]; sd[0] = s_b0[slot]; sd[1] = s_b1[slot]; rb = rb_b; lpos = B.row_pos;
            } else {
                rec.count = s_cnt[slot]; sd[0] = s_s0[slot]; sd[1] = s_s1[slot]; rb = rb_f; lpos = F.row_pos;
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (sd[q] == SEED_NONE) { rec.qpos[q] = 0xFFFF; rec.tpos[q] = 0xFFFF; continue; }
                const int64_t t = (int64_t)(sd[q] >> 16);
                rec.qpos[q] = lpos[rb + t];
                rec.tpos[q] = (uint16_t)(sd[q] & 0xFFFF);
            }
            tmp_out[it.out_off + out_n + r] = rec;
        }
        out_n += nv;
        n_rec += (unsigned long long)nv;
        __syncthreads();                 // the table is cleared for the next range
        a = z;
    }
    if (threadIdx.x == 0) {
        item_count[blockIdx.x] = out_n;
        if (stats) atomicAdd(&stats[2], n_rec);
    }
}

__global__ void k_concat(const pastis_cand *tmp, const int64_t *src_off, const int64_t *dst_off, const int64_t *cnt,
                         int64_t n_items, pastis_cand *out) {
    // one warp per item
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_items) return;
    const int64_t src = src_off[w], dst = dst_off[w], c = cnt[w];
    for (int64_t r = lane; r < c; r += 32) out[dst + r] = tmp[src + r];
}

size_t table_bytes(int tsize, bool subs) {
    return subs ? (size_t)tsize * (4 * 8 + 3 * 4 + 2 * 4) : (size_t)tsize * (2 * 8 + 2 * 4 + 2 * 4);
}

}  // namespace

cudaError_t spgemm_set_smem_limit(size_t bytes) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_spgemm_rows<true>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_spgemm_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(bytes - fa.sharedSizeBytes));
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_spgemm_rows<false>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_spgemm_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(bytes - fa.sharedSizeBytes));
    return e;
}

// The product driver.  Self mode (DB == nullptr): rows of A against A's postings,
// columns j > i.  Query mode: rows of A (the queries) against the postings of DB,
// every column j of DB (exact k-mers only).
static pastis_status overlap_impl(pastis_ctx *ctx, const pastis_kmat *A, const pastis_kmat *DB,
                                  const pastis_params *params, int32_t row_begin, int32_t row_end, pastis_cand *d_out,
                                  int64_t capacity, int64_t *n_out) {
    if (!ctx || !A || !n_out || capacity < 0) return PASTIS_ERR_INVALID_ARG;
    if (row_begin < 0 || row_end < row_begin || row_end > A->n_rows) return PASTIS_ERR_INVALID_ARG;
    pastis_status s = check_params(params);
    if (s != PASTIS_OK) return s;
    if (A->k != params->k || A->n_rows < 0) return PASTIS_ERR_INVALID_ARG;
    const bool self = DB == nullptr;
    if (!self && (DB->k != params->k || params->m_subs != 0)) return self ? PASTIS_ERR_INVALID_ARG : PASTIS_ERR_UNSUPPORTED;
    cudaStream_t st = ctx->stream;
    const int32_t n = A->n_rows;
    const int32_t n_cols = self ? n : DB->n_rows;
    const bool subs = params->m_subs > 0;
    const uint32_t mh = params_matrix_hash(params);
    const void *key_b = self ? nullptr : (const void *)DB->col_ptr;

    // a kept result for the same inputs: copy it (two-phase size protocol)
    if (ctx->spg_valid && ctx->spg_key_b == key_b && ctx->spg_key_a == (const void *)A->row_ptr && ctx->spg_key_nnz == A->nnz &&
        ctx->spg_key_m == params->m_subs && ctx->spg_key_min == params->min_shared &&
        ctx->spg_key_k == params->k && ctx->spg_key_mat_hash == (subs ? mh : 0u) &&
        ctx->spg_key_r0 == row_begin && ctx->spg_key_r1 == row_end) {
        *n_out = ctx->spg_n;
        if (capacity < ctx->spg_n) return PASTIS_ERR_CAPACITY;
        if (ctx->spg_n > 0) {
            if (!d_out) return PASTIS_ERR_INVALID_ARG;
            PASTIS_CUDA_TRY(cudaMemcpyAsync(d_out, ctx->ws[WS_SPG_RESULT], sizeof(pastis_cand) * ctx->spg_n,
                                            cudaMemcpyDeviceToDevice, st));
            PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
        }
        return PASTIS_OK;
    }
    ctx->spg_valid = 0;
    if ((self && n < 2) || (!self && (n < 1 || n_cols < 1)) || A->nnz == 0 || (!self && DB->nnz == 0)) {
        *n_out = 0;
        return PASTIS_OK;
    }

    operand F, Bop;
    F.row_ptr = A->row_ptr; F.row_code = A->row_code; F.row_pos = A->row_pos;
    const pastis_kmat *C = self ? A : DB;
    F.col_ptr = C->col_ptr; F.col_seq = C->col_seq; F.col_pos = C->col_pos;
    Bop = F;
    if (subs) {
        as_matrix AS;
        s = build_as(ctx, A, params, &AS);
        if (s != PASTIS_OK) return s;
        // forward: rows of AS against the postings of A
        F.row_ptr = AS.row_ptr; F.row_code = AS.row_code; F.row_pos = AS.row_pos;
        // backward: rows of A against the postings of AS
        Bop.col_ptr = AS.col_ptr; Bop.col_seq = AS.col_seq; Bop.col_pos = AS.col_pos;
    }

    // rows that can form products: left entries per row from the row pointers
    const int32_t nr = row_end - row_begin;
    std::vector<int64_t> rpf((size_t)nr + 1), rpb((size_t)nr + 1);
    PASTIS_CUDA_TRY(cudaMemcpyAsync(rpf.data(), F.row_ptr + row_begin, sizeof(int64_t) * (nr + 1),
                                    cudaMemcpyDeviceToHost, st));
    if (subs)
        PASTIS_CUDA_TRY(cudaMemcpyAsync(rpb.data(), Bop.row_ptr + row_begin, sizeof(int64_t) * (nr + 1),
                                        cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int32_t> rows;
    std::vector<int64_t> ent_off;
    rows.reserve((size_t)nr);
    ent_off.reserve((size_t)nr + 1);
    int64_t n_ent = 0;
    for (int32_t r = 0; r < nr; ++r) {
        const int32_t i = row_begin + r;
        if ((self ? i + 1 : 0) >= n_cols) continue;
        const int64_t ne = (rpf[r + 1] - rpf[r]) + (subs ? rpb[r + 1] - rpb[r] : 0);
        if (ne == 0) continue;
        rows.push_back(i);
        ent_off.push_back(n_ent);
        n_ent += ne;
    }
    const int64_t ni = (int64_t)rows.size();
    if (ni == 0) {
        *n_out = 0;
        return PASTIS_OK;
    }

    // cursors of every row (exact products per row)
    cursors cur;
    int32_t *d_rows;
    PASTIS_WS(d_rows, ctx, WS_SPG_ROWWORK, (sizeof(int32_t) + 3 * sizeof(int64_t)) * (size_t)ni + 64);
    int64_t *d_eoff = (int64_t *)(((uintptr_t)(d_rows + ni) + 7) & ~(uintptr_t)7);
    int64_t *d_nact = d_eoff + ni;
    int64_t *d_nprod = d_nact + ni;
    char *cbuf;
    PASTIS_WS(cbuf, ctx, WS_SPG_CURSORS, (sizeof(int32_t) * 2 + sizeof(int64_t) * 2) * (size_t)n_ent + 64);
    cur.x = (int64_t *)cbuf;
    cur.pe = cur.x + n_ent;
    cur.nj = (int32_t *)(cur.pe + n_ent);
    cur.t = (uint32_t *)(cur.nj + n_ent);
    PASTIS_CUDA_TRY(cudaMemcpyAsync(d_rows, rows.data(), sizeof(int32_t) * ni, cudaMemcpyHostToDevice, st));
    PASTIS_CUDA_TRY(cudaMemcpyAsync(d_eoff, ent_off.data(), sizeof(int64_t) * ni, cudaMemcpyHostToDevice, st));
    unsigned long long *stats = ctx->prof_on ? ctx->d_stats : nullptr;
    prof_begin(ctx, "spgemm_cursors");
    k_spgemm_cursors<<<(unsigned)ceil_div64(ni * 32, CUR_THREADS), CUR_THREADS, 0, st>>>(
        F, Bop, subs ? 1 : 0, self ? 1 : 0, d_rows, d_eoff, (int32_t)ni, cur, d_nact, d_nprod, stats);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    std::vector<int64_t> nact((size_t)ni), nprod((size_t)ni);
    PASTIS_CUDA_TRY(cudaMemcpyAsync(nact.data(), d_nact, sizeof(int64_t) * ni, cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaMemcpyAsync(nprod.data(), d_nprod, sizeof(int64_t) * ni, cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));

    // plan: rows with products, each with a table size and a starting number of column
    // ranges (distinct j <= products; ranges sized for a table half full)
    int tmax = 1 << 14;
    while (tmax > 64 && table_bytes(tmax, subs) + 64 > ctx->smem_optin) tmax >>= 1;
    int tl_max = 0;
    while ((1 << tl_max) < tmax) ++tl_max;
    struct plan_row { row_item it; int tlog; int64_t order; };
    std::vector<plan_row> plan;
    plan.reserve((size_t)ni);
    int64_t tmp_total = 0;
    for (int64_t r = 0; r < ni; ++r) {
        if (nprod[r] == 0) continue;
        const int32_t i = rows[r];
        const int64_t width = (int64_t)n_cols - (self ? i + 1 : 0);
        const int64_t est = std::min<int64_t>(nprod[r], width);
        plan_row p;
        p.it.i = i;
        p.it.ent_off = ent_off[r];
        p.it.n_act = nact[r];
        p.it.out_cap = est;
        p.order = r;
        if (est * 4 <= (int64_t)tmax * 3) {
            int tl = 6;
            while ((1ll << tl) * 3 < est * 4) ++tl;
            p.tlog = tl;
            p.it.pieces = 1;
        } else {
            p.tlog = tl_max;
            p.it.pieces = (int32_t)std::min<int64_t>(width, ceil_div64(est * 2, tmax));
        }
        p.it.out_off = tmp_total;
        tmp_total += est;
        plan.push_back(p);
    }
    const int64_t np = (int64_t)plan.size();
    int64_t total = 0;
    pastis_cand *result = nullptr;
    if (np > 0) {
        std::stable_sort(plan.begin(), plan.end(), [](const plan_row &a, const plan_row &b) { return a.tlog < b.tlog; });
        std::vector<row_item> wi((size_t)np);
        for (int64_t x = 0; x < np; ++x) wi[x] = plan[x].it;
        row_item *d_items;
        PASTIS_WS(d_items, ctx, WS_SPG_BIN, sizeof(row_item) * np + (sizeof(int64_t) + sizeof(int)) * np + 64);
        int64_t *d_cnt = (int64_t *)(d_items + np);
        int *d_err = (int *)(d_cnt + np);
        pastis_cand *tmp;
        PASTIS_WS(tmp, ctx, WS_SPG_TMP, sizeof(pastis_cand) * (size_t)(tmp_total + 1));
        PASTIS_CUDA_TRY(cudaMemcpyAsync(d_items, wi.data(), sizeof(row_item) * np, cudaMemcpyHostToDevice, st));
        PASTIS_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int) * np, st));
        int64_t x0 = 0;
        while (x0 < np) {
            int64_t x1 = x0;
            while (x1 < np && plan[x1].tlog == plan[x0].tlog) ++x1;
            const int tsize = 1 << plan[x0].tlog;
            const size_t shm = table_bytes(tsize, subs);
            for (int64_t g0 = x0; g0 < x1; g0 += 65535) {
                const int64_t g1 = std::min<int64_t>(x1, g0 + 65535);
                prof_begin(ctx, "spgemm_rows");
                const int nth = spg_threads_for(tsize);
                if (subs)
                    k_spgemm_rows<true><<<(unsigned)(g1 - g0), nth, shm, st>>>(
                        F, Bop, d_items + g0, tsize, params->min_shared, self ? 1 : 0, n_cols, cur, tmp, d_cnt + g0,
                        d_err + g0, stats);
                else
                    k_spgemm_rows<false><<<(unsigned)(g1 - g0), nth, shm, st>>>(
                        F, Bop, d_items + g0, tsize, params->min_shared, self ? 1 : 0, n_cols, cur, tmp, d_cnt + g0,
                        d_err + g0, stats);
                PASTIS_LAUNCHED(ctx);
                prof_end(ctx);
            }
            x0 = x1;
        }
        std::vector<int64_t> hc((size_t)np);
        std::vector<int> he((size_t)np);
        PASTIS_CUDA_TRY(cudaMemcpyAsync(hc.data(), d_cnt, sizeof(int64_t) * np, cudaMemcpyDeviceToHost, st));
        PASTIS_CUDA_TRY(cudaMemcpyAsync(he.data(), d_err, sizeof(int) * np, cudaMemcpyDeviceToHost, st));
        PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
        // slices in row order
        std::vector<int64_t> ord((size_t)np);
        for (int64_t x = 0; x < np; ++x) {
            if (he[x]) return PASTIS_ERR_INTERNAL;
            ord[x] = x;
        }
        std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return plan[a].order < plan[b].order; });
        std::vector<int64_t> src, dst, cnt;
        for (int64_t x : ord) {
            if (hc[x] == 0) continue;
            src.push_back(plan[x].it.out_off);
            dst.push_back(total);
            cnt.push_back(hc[x]);
            total += hc[x];
        }
        PASTIS_WS(result, ctx, WS_SPG_RESULT, sizeof(pastis_cand) * (size_t)(total + 1));
        const int64_t nk = (int64_t)src.size();
        if (nk > 0) {
            int64_t *d_src;
            PASTIS_WS(d_src, ctx, WS_SPG_ROWOFF, 3 * sizeof(int64_t) * (size_t)nk + 64);
            int64_t *d_dst = d_src + nk;
            int64_t *d_c = d_dst + nk;
            PASTIS_CUDA_TRY(cudaMemcpyAsync(d_src, src.data(), sizeof(int64_t) * nk, cudaMemcpyHostToDevice, st));
            PASTIS_CUDA_TRY(cudaMemcpyAsync(d_dst, dst.data(), sizeof(int64_t) * nk, cudaMemcpyHostToDevice, st));
            PASTIS_CUDA_TRY(cudaMemcpyAsync(d_c, cnt.data(), sizeof(int64_t) * nk, cudaMemcpyHostToDevice, st));
            prof_begin(ctx, "spgemm_concat");
            k_concat<<<(unsigned)ceil_div64(nk * 32, 256), 256, 0, st>>>(tmp, d_src, d_dst, d_c, nk, result);
            PASTIS_LAUNCHED(ctx);
            prof_end(ctx);
            PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
        }
    }
    ctx->spg_valid = 1;
    ctx->spg_n = total;
    ctx->spg_key_a = (const void *)A->row_ptr;
    ctx->spg_key_nnz = A->nnz;
    ctx->spg_key_m = params->m_subs;
    ctx->spg_key_min = params->min_shared;
    ctx->spg_key_k = params->k;
    ctx->spg_key_mat_hash = subs ? mh : 0u;
    ctx->spg_key_r0 = row_begin;
    ctx->spg_key_r1 = row_end;
    ctx->spg_key_b = key_b;
    *n_out = total;
    if (capacity < total) return PASTIS_ERR_CAPACITY;
    if (total > 0) {
        if (!d_out) return PASTIS_ERR_INVALID_ARG;
        PASTIS_CUDA_TRY(cudaMemcpyAsync(d_out, result, sizeof(pastis_cand) * total, cudaMemcpyDeviceToDevice, st));
        PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return PASTIS_OK;
}

extern "C" pastis_status pastis_overlap_spgemm_rows(pastis_ctx *ctx, const pastis_kmat *A,
                                                    const pastis_params *params, int32_t row_begin, int32_t row_end,
                                                    pastis_cand *d_out, int64_t capacity, int64_t *n_out) {
    return overlap_impl(ctx, A, nullptr, params, row_begin, row_end, d_out, capacity, n_out);
}

extern "C" pastis_status pastis_overlap_spgemm(pastis_ctx *ctx, const pastis_kmat *A, const pastis_params *params,
                                               pastis_cand *d_out, int64_t capacity, int64_t *n_out) {
    if (!A) return PASTIS_ERR_INVALID_ARG;
    return overlap_impl(ctx, A, nullptr, params, 0, A->n_rows, d_out, capacity, n_out);
}

extern "C" pastis_status pastis_query_overlap(pastis_ctx *ctx, const pastis_kmat *Q, const pastis_kmat *DB,
                                              const pastis_params *params, pastis_cand *d_out, int64_t capacity,
                                              int64_t *n_out) {
    if (!Q || !DB) return PASTIS_ERR_INVALID_ARG;
    return overlap_impl(ctx, Q, DB, params, 0, Q->n_rows, d_out, capacity, n_out);
}
