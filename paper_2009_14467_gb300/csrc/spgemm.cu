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
// Row-wise hash SpGEMM.  A work item is a row i and a column range [J0, J1) of j > i.
// One CTA owns an item and a hash table in shared memory keyed by j; each left entry
// (k-mer t of row i) walks its posting list (sorted by sequence, so the range start is
// found by binary search) and for every j inserts: count += 1 and the seed
// t << 16 | pos_j into a two-smallest pair with the atomicMin swap
//     old = atomicMin(s0, v);  atomicMin(s1, max(old, v))
// which leaves s0, s1 = the two smallest values whatever the arrival order.  Row
// entries are in ascending code order, so the smallest t is the smallest code.  The
// CTA then compacts the entries that pass min_shared, sorts them by j (bitonic), and
// writes records to a per-item slice; a final pass concatenates the slices in (i, j)
// order.  Rows whose product bound exceeds a table are split into column ranges by
// the host; a range that still overflows is flagged and split again.
#include <algorithm>
#include <vector>

#include "internal.cuh"

struct as_matrix {
    int64_t nnz;
    int64_t *row_ptr;
    uint32_t *row_code;
    uint16_t *row_pos;
    uint32_t *col_ptr;
    int32_t *col_seq;
    uint16_t *col_pos;
};
pastis_status build_as(pastis_ctx *ctx, const pastis_kmat *A, const pastis_params *p, as_matrix *out);

namespace {

constexpr int SPG_THREADS = 256;
constexpr uint64_t SEED_NONE = ~0ull;

struct operand {          // one side of the product: left rows and right posting lists
    const int64_t *row_ptr;
    const uint32_t *row_code;
    const uint16_t *row_pos;
    const uint32_t *col_ptr;
    const int32_t *col_seq;
    const uint16_t *col_pos;
};

struct work_item {
    int32_t i;
    int32_t j0, j1;       // column range [j0, j1)
    int32_t first;        // 1 when j0 is the row's first column (its left entries are counted there)
    int64_t out_off;      // slice in the temporary record buffer
    int64_t out_cap;
};

// Upper bound of the products of row i over j > i: posting lengths of its entries.
__global__ void k_row_bound(operand L, int32_t n, int64_t *bound) {
    int32_t i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    int64_t acc = 0;
    for (int64_t t = L.row_ptr[i] + lane; t < L.row_ptr[i + 1]; t += 32) {
        uint32_t c = L.row_code[t];
        acc += (int64_t)(L.col_ptr[c + 1] - L.col_ptr[c]);
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    if (lane == 0) bound[i] = acc;
}

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

// Inserts every product of one orientation into the table.  Returns false on overflow.
template <bool TWO>
__device__ void insert_side(const operand &L, int32_t i, int32_t j0, int32_t j1, int32_t *s_key,
                            uint32_t *s_cnt, unsigned long long *s_s0, unsigned long long *s_s1, int tsize,
                            int *s_overflow, unsigned long long &n_left, unsigned long long &n_prod) {
    const int64_t rb = L.row_ptr[i], re = L.row_ptr[i + 1];
    for (int64_t t = rb + threadIdx.x; t < re; t += blockDim.x) {
        const uint32_t c = L.row_code[t];
        const int64_t pb = L.col_ptr[c], pe = L.col_ptr[c + 1];
        int64_t x = lower_bound_seq(L.col_seq, pb, pe, j0);
        const unsigned long long tv = (unsigned long long)(t - rb) << 16;
        ++n_left;
        for (; x < pe; ++x) {
            const int32_t j = L.col_seq[x];
            if (j >= j1) break;
            ++n_prod;
            uint32_t slot = hash_j(j) & (uint32_t)(tsize - 1);
            int probes = 0;
            for (;;) {
                int32_t prev = atomicCAS(&s_key[slot], -1, j);
                if (prev == -1 || prev == j) break;
                slot = (slot + 1) & (uint32_t)(tsize - 1);
                if (++probes >= tsize) { *s_overflow = 1; return; }
            }
            atomicAdd(&s_cnt[slot], 1u);
            const unsigned long long v = tv | (unsigned long long)L.col_pos[x];
            const unsigned long long old = atomicMin(&s_s0[slot], v);
            atomicMin(&s_s1[slot], old > v ? old : v);
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

// One CTA per work item.  SUBS: two orientations per entry (fwd = (AS)_i A_j,
// bwd = A_i (AS)_j).  Shared memory: key[T], cnt[T], s0[T], s1[T] (+ cnt_b, s0_b, s1_b),
// then sort scratch key[T], val[T].
template <bool SUBS>
__global__ void __launch_bounds__(SPG_THREADS) k_spgemm_items(operand F, operand B, const work_item *items,
                                                              int tsize, int32_t min_shared,
                                                              pastis_cand *tmp_out, int64_t *item_count,
                                                              int *item_overflow, unsigned long long *stats) {
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

    const work_item it = items[blockIdx.x];
    for (int x = threadIdx.x; x < tsize; x += blockDim.x) {
        s_key[x] = -1;
        s_cnt[x] = 0;
        s_s0[x] = SEED_NONE;
        s_s1[x] = SEED_NONE;
        if (SUBS) { s_cntb[x] = 0; s_b0[x] = SEED_NONE; s_b1[x] = SEED_NONE; }
    }
    if (threadIdx.x == 0) { s_overflow = 0; s_nvalid = 0; }
    __syncthreads();
    unsigned long long n_left = 0, n_prod = 0;
    insert_side<SUBS>(F, it.i, it.j0, it.j1, s_key, s_cnt, s_s0, s_s1, tsize, &s_overflow, n_left, n_prod);
    if (SUBS) insert_side<SUBS>(B, it.i, it.j0, it.j1, s_key, s_cntb, s_b0, s_b1, tsize, &s_overflow, n_left, n_prod);
    __syncthreads();
    if (s_overflow) {
        if (threadIdx.x == 0) { item_overflow[blockIdx.x] = 1; item_count[blockIdx.x] = 0; }
        return;
    }
    // compact passing entries
    for (int x = threadIdx.x; x < tsize; x += blockDim.x) {
        if (s_key[x] < 0) continue;
        uint32_t c = s_cnt[x];
        if (SUBS && s_cntb[x] > c) c = s_cntb[x];
        if ((int64_t)c < (int64_t)min_shared) continue;
        int r = atomicAdd(&s_nvalid, 1);
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
    if (nv > it.out_cap) {   // cannot happen with the capacities the planner sets
        if (threadIdx.x == 0) { item_overflow[blockIdx.x] = 1; item_count[blockIdx.x] = 0; }
        return;
    }
    const int64_t rb_f = F.row_ptr[it.i];
    const int64_t rb_b = SUBS ? B.row_ptr[it.i] : 0;
    for (int r = threadIdx.x; r < nv; r += blockDim.x) {
        const int slot = (int)s_sv[r];
        pastis_cand rec;
        rec.i = it.i;
        rec.j = (int32_t)s_sk[r];
        bool use_b = SUBS && (s_cntb[slot] > s_cnt[slot]);
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
            int64_t t = (int64_t)(sd[q] >> 16);
            rec.qpos[q] = lpos[rb + t];
            rec.tpos[q] = (uint16_t)(sd[q] & 0xFFFF);
        }
        tmp_out[it.out_off + r] = rec;
    }
    if (threadIdx.x == 0) item_count[blockIdx.x] = nv;
    if (stats) {                     // work of the items that completed (profiling only)
        for (int x = 16; x > 0; x >>= 1) {
            n_left += __shfl_xor_sync(0xffffffffu, n_left, x);
            n_prod += __shfl_xor_sync(0xffffffffu, n_prod, x);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&stats[0], n_prod);
            if (it.first) atomicAdd(&stats[1], n_left);   // each left entry once per row
            if (threadIdx.x == 0) atomicAdd(&stats[2], (unsigned long long)nv);
        }
    }
}

__global__ void k_concat(const pastis_cand *tmp, const work_item *items, const int64_t *item_count,
                         const int64_t *item_dst, int64_t n_items, pastis_cand *out) {
    // one warp per item
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_items) return;
    const int64_t src = items[w].out_off, dst = item_dst[w], cnt = item_count[w];
    for (int64_t r = lane; r < cnt; r += 32) out[dst + r] = tmp[src + r];
}

size_t table_bytes(int tsize, bool subs) {
    return subs ? (size_t)tsize * (4 * 8 + 3 * 4 + 2 * 4) : (size_t)tsize * (2 * 8 + 2 * 4 + 2 * 4);
}

}  // namespace

// The product driver.  Self mode (DB == nullptr): rows of A against A's postings,
// columns j > i.  Query mode: rows of A (the queries) against the postings of DB,
// every column j of DB (exact k-mers only).
cudaError_t spgemm_set_smem_limit(size_t bytes) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_spgemm_items<true>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_spgemm_items<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(bytes - fa.sharedSizeBytes));
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_spgemm_items<false>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_spgemm_items<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(bytes - fa.sharedSizeBytes));
    return e;
}

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

    // per-row product bounds
    int64_t *bound;
    PASTIS_WS(bound, ctx, WS_SPG_ROWWORK, sizeof(int64_t) * 2 * (size_t)n);
    int64_t *bound_b = bound + n;
    prof_begin(ctx, "spgemm_bound");
    k_row_bound<<<(unsigned)ceil_div64(n, 8), 256, 0, st>>>(F, n, bound);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    if (subs) {
        prof_begin(ctx, "spgemm_bound");
        k_row_bound<<<(unsigned)ceil_div64(n, 8), 256, 0, st>>>(Bop, n, bound_b);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    std::vector<int64_t> hb((size_t)n * (subs ? 2 : 1));
    PASTIS_CUDA_TRY(cudaMemcpyAsync(hb.data(), bound, sizeof(int64_t) * hb.size(), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));

    // table size limit from shared memory
    int tmax = 1 << 14;
    while (tmax > 64 && table_bytes(tmax, subs) + 64 > ctx->smem_optin) tmax >>= 1;

    // plan: items by (i, column range), each with a table size
    struct plan_item { int32_t i, j0, j1; int tlog; int64_t cap; };
    std::vector<plan_item> plan;
    plan.reserve((size_t)n);
    for (int32_t i = row_begin; i < row_end; ++i) {
        const int32_t jlo = self ? i + 1 : 0;
        if (jlo >= n_cols) continue;
        int64_t b = hb[i] + (subs ? hb[(size_t)n + i] : 0);
        int64_t width = n_cols - jlo;
        int64_t est = std::min(b, width);
        if (est <= 0) continue;
        if (est * 4 <= (int64_t)tmax * 3) {
            int tl = 6;
            while ((1ll << tl) * 3 < est * 4) ++tl;
            plan.push_back({i, jlo, n_cols, tl, est});
        } else {
            int tl = 0;
            while ((1 << tl) < tmax) ++tl;
            int64_t pieces = ceil_div64(est * 2, tmax);
            for (int64_t q = 0; q < pieces; ++q) {
                int32_t a = (int32_t)(jlo + (width * q) / pieces);
                int32_t z = (int32_t)(jlo + (width * (q + 1)) / pieces);
                if (z > a) plan.push_back({i, a, z, tl, std::min<int64_t>(std::min<int64_t>(b, z - a), tmax)});
            }
        }
    }

    // upper bound of the records: distinct j per row
    int64_t ubound = 0;
    for (int32_t i = row_begin; i < row_end; ++i) {
        const int32_t jlo = self ? i + 1 : 0;
        if (jlo < n_cols) ubound += std::min<int64_t>(hb[i] + (subs ? hb[(size_t)n + i] : 0), (int64_t)(n_cols - jlo));
    }
    pastis_cand *result;
    PASTIS_WS(result, ctx, WS_SPG_RESULT, sizeof(pastis_cand) * (size_t)(ubound + 1));

    // run all pending items grouped by table size; split the ones that overflow and rerun
    struct round_out { std::vector<plan_item> items; std::vector<int64_t> offs; std::vector<int64_t> cnts; };
    std::vector<round_out> rounds_out;
    int64_t tmp_total = 0;
    int rounds = 0;
    std::vector<plan_item> pending = plan;
    while (!pending.empty()) {
        if (++rounds > 24) return PASTIS_ERR_INTERNAL;
        std::stable_sort(pending.begin(), pending.end(),
                         [](const plan_item &a, const plan_item &b) { return a.tlog < b.tlog; });
        const int64_t ni = (int64_t)pending.size();
        std::vector<work_item> wi((size_t)ni);
        int64_t off = 0;
        for (int64_t x = 0; x < ni; ++x) {
            wi[x].i = pending[x].i; wi[x].j0 = pending[x].j0; wi[x].j1 = pending[x].j1;
            wi[x].first = pending[x].j0 == (self ? pending[x].i + 1 : 0);
            wi[x].out_off = off; wi[x].out_cap = pending[x].cap;
            off += pending[x].cap;
        }
        work_item *d_items;
        PASTIS_WS(d_items, ctx, WS_SPG_BIN, sizeof(work_item) * ni + sizeof(int64_t) * 3 * ni + 64);
        int64_t *d_cnt = (int64_t *)(d_items + ni);
        int *d_ovf = (int *)(d_cnt + ni);
        pastis_cand *tmp;
        PASTIS_WS(tmp, ctx, WS_SPG_TMP, sizeof(pastis_cand) * (size_t)(off + 1));
        PASTIS_CUDA_TRY(cudaMemcpyAsync(d_items, wi.data(), sizeof(work_item) * ni, cudaMemcpyHostToDevice, st));
        PASTIS_CUDA_TRY(cudaMemsetAsync(d_ovf, 0, sizeof(int) * ni, st));
        int64_t x0 = 0;
        while (x0 < ni) {
            int64_t x1 = x0;
            while (x1 < ni && pending[x1].tlog == pending[x0].tlog) ++x1;
            const int tsize = 1 << pending[x0].tlog;
            const size_t shm = table_bytes(tsize, subs);
            for (int64_t g0 = x0; g0 < x1; g0 += 65535) {
                int64_t g1 = std::min<int64_t>(x1, g0 + 65535);
                prof_begin(ctx, "spgemm_items");
                if (subs)
                    k_spgemm_items<true><<<(unsigned)(g1 - g0), SPG_THREADS, shm, st>>>(
                        F, Bop, d_items + g0, tsize, params->min_shared, tmp, d_cnt + g0, d_ovf + g0,
                        ctx->prof_on ? ctx->d_stats : nullptr);
                else
                    k_spgemm_items<false><<<(unsigned)(g1 - g0), SPG_THREADS, shm, st>>>(
                        F, Bop, d_items + g0, tsize, params->min_shared, tmp, d_cnt + g0, d_ovf + g0,
                        ctx->prof_on ? ctx->d_stats : nullptr);
                PASTIS_LAUNCHED(ctx);
                prof_end(ctx);
            }
            x0 = x1;
        }
        std::vector<int64_t> hc((size_t)ni);
        std::vector<int> ho((size_t)ni);
        PASTIS_CUDA_TRY(cudaMemcpyAsync(hc.data(), d_cnt, sizeof(int64_t) * ni, cudaMemcpyDeviceToHost, st));
        PASTIS_CUDA_TRY(cudaMemcpyAsync(ho.data(), d_ovf, sizeof(int) * ni, cudaMemcpyDeviceToHost, st));
        PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
        round_out ro;
        std::vector<plan_item> next;
        int tl_max = 0;
        while ((1 << tl_max) < tmax) ++tl_max;
        for (int64_t x = 0; x < ni; ++x) {
            if (ho[x]) {
                // grow the table to the maximum first, then halve the column range
                plan_item p = pending[x];
                if (p.tlog < tl_max) {
                    p.tlog = tl_max;
                    p.cap = std::min<int64_t>((int64_t)p.j1 - p.j0, (int64_t)tmax);
                    next.push_back(p);
                    continue;
                }
                if (p.j1 - p.j0 < 2) return PASTIS_ERR_INTERNAL;
                int32_t mid = p.j0 + (p.j1 - p.j0) / 2;
                next.push_back({p.i, p.j0, mid, p.tlog, std::min<int64_t>((int64_t)tmax, mid - p.j0)});
                next.push_back({p.i, mid, p.j1, p.tlog, std::min<int64_t>((int64_t)tmax, p.j1 - mid)});
                continue;
            }
            if (hc[x] > 0) {
                ro.items.push_back(pending[x]);
                ro.offs.push_back(wi[x].out_off);
                ro.cnts.push_back(hc[x]);
            }
        }
        // gather this round's slices, in (i, j0) order, into the result area after the
        // earlier rounds
        const int64_t nk = (int64_t)ro.items.size();
        if (nk > 0) {
            std::vector<int64_t> ord((size_t)nk);
            for (int64_t x = 0; x < nk; ++x) ord[x] = x;
            std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
                return ro.items[a].i != ro.items[b].i ? ro.items[a].i < ro.items[b].i : ro.items[a].j0 < ro.items[b].j0;
            });
            round_out sorted;
            for (int64_t x : ord) {
                sorted.items.push_back(ro.items[x]);
                sorted.offs.push_back(ro.offs[x]);
                sorted.cnts.push_back(ro.cnts[x]);
            }
            ro = sorted;
            std::vector<work_item> src((size_t)nk);
            std::vector<int64_t> dst((size_t)nk);
            for (int64_t x = 0; x < nk; ++x) {
                src[x].out_off = ro.offs[x];
                dst[x] = tmp_total;
                ro.offs[x] = tmp_total;   // now the position in the result area
                tmp_total += ro.cnts[x];
            }
            if (tmp_total > ubound) return PASTIS_ERR_INTERNAL;
            work_item *d_src;
            PASTIS_WS(d_src, ctx, WS_SPG_ROWOFF, (sizeof(work_item) + 2 * sizeof(int64_t)) * (size_t)nk + 64);
            int64_t *d_dst = (int64_t *)(d_src + nk);
            int64_t *d_c = d_dst + nk;
            PASTIS_CUDA_TRY(cudaMemcpyAsync(d_src, src.data(), sizeof(work_item) * nk, cudaMemcpyHostToDevice, st));
            PASTIS_CUDA_TRY(cudaMemcpyAsync(d_dst, dst.data(), sizeof(int64_t) * nk, cudaMemcpyHostToDevice, st));
            PASTIS_CUDA_TRY(cudaMemcpyAsync(d_c, ro.cnts.data(), sizeof(int64_t) * nk, cudaMemcpyHostToDevice, st));
            prof_begin(ctx, "spgemm_concat");
            k_concat<<<(unsigned)ceil_div64(nk * 32, 256), 256, 0, st>>>(tmp, d_src, d_c, d_dst, nk, result);
            PASTIS_LAUNCHED(ctx);
            prof_end(ctx);
            PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
        }
        rounds_out.push_back(ro);
        pending.swap(next);
    }
    // final order: all kept slices sorted by (i, j0); a single round is already in order
    int64_t total = tmp_total;
    if (rounds_out.size() > 1 && total > 0) {
        struct sl { int32_t i, j0; int64_t off, cnt; };
        std::vector<sl> all;
        for (auto &ro : rounds_out)
            for (size_t x = 0; x < ro.items.size(); ++x) all.push_back({ro.items[x].i, ro.items[x].j0, ro.offs[x], ro.cnts[x]});
        std::sort(all.begin(), all.end(), [](const sl &a, const sl &b) { return a.i != b.i ? a.i < b.i : a.j0 < b.j0; });
        const int64_t nk = (int64_t)all.size();
        std::vector<work_item> src((size_t)nk);
        std::vector<int64_t> dst((size_t)nk), cnt((size_t)nk);
        int64_t acc = 0;
        for (int64_t x = 0; x < nk; ++x) { src[x].out_off = all[x].off; dst[x] = acc; cnt[x] = all[x].cnt; acc += cnt[x]; }
        pastis_cand *tmp2;
        PASTIS_WS(tmp2, ctx, WS_SPG_TMP, sizeof(pastis_cand) * (size_t)(total + 1));
        PASTIS_CUDA_TRY(cudaMemcpyAsync(tmp2, result, sizeof(pastis_cand) * total, cudaMemcpyDeviceToDevice, st));
        work_item *d_src;
        PASTIS_WS(d_src, ctx, WS_SPG_ROWOFF, (sizeof(work_item) + 2 * sizeof(int64_t)) * (size_t)nk + 64);
        int64_t *d_dst = (int64_t *)(d_src + nk);
        int64_t *d_c = d_dst + nk;
        PASTIS_CUDA_TRY(cudaMemcpyAsync(d_src, src.data(), sizeof(work_item) * nk, cudaMemcpyHostToDevice, st));
        PASTIS_CUDA_TRY(cudaMemcpyAsync(d_dst, dst.data(), sizeof(int64_t) * nk, cudaMemcpyHostToDevice, st));
        PASTIS_CUDA_TRY(cudaMemcpyAsync(d_c, cnt.data(), sizeof(int64_t) * nk, cudaMemcpyHostToDevice, st));
        prof_begin(ctx, "spgemm_concat");
        k_concat<<<(unsigned)ceil_div64(nk * 32, 256), 256, 0, st>>>(tmp2, d_src, d_c, d_dst, nk, result);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
        PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
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
