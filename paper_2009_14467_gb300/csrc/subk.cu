// a4-a5: substitute k-mers (the matrix S) and the product AS.
//
// Sec. IV-B: the expense of replacing base a by b is C[a][a] - C[a][b] (the matrix
// E = Sort(Diag(C) - C)); a k-mer's distance from a root is the sum of its per-position
// expenses.  Row r of S holds r itself (distance 0) and the m k-mers q != r nearest to
// r, ties broken by the smaller code.  Alg. 1-3 reach that set with a best-first
// search over min-max heaps; on the GPU each thread owns one root and finds it in two
// fixed-size phases instead:
//   1. the number of k-mers at every distance, as a convolution over positions of the
//      per-position expense histograms; it yields the cut distance D* (the first
//      distance at which at least m k-mers q != r are reached) and how many of the
//      ties at D* are taken;
//   2. one depth-first walk of the k-mer tree in code order, pruned at D*: every
//      k-mer closer than D* and the first `quota` ones at D* are written straight to
//      their sorted slot, slot = (number of k-mers closer than it) + (its rank among
//      equal distances in code order).
// Sec. IV-C: AS(i, s) keeps the start of the k-mer of sequence i nearest to s (the
// smaller start on ties).  AS is expanded from the rows of A and S, radix-sorted by s
// (stable, so sequences stay ascending), reduced to one entry per (s, i), and sorted
// again by sequence for its CSR view.
#include <string.h>

#include "internal.cuh"

namespace {

constexpr int SUBK_DLIM = 64;     // shifted distances handled (see check_params bounds)
constexpr int SUBK_THREADS = 128;

__global__ void __launch_bounds__(SUBK_THREADS) k_subkmers(const uint32_t *__restrict__ roots, int64_t n_roots,
                                                           int k, int m, const int8_t *__restrict__ gmat,
                                                           uint32_t *__restrict__ out_code,
                                                           int32_t *__restrict__ out_dist, int *err) {
    __shared__ int s_exp[PASTIS_NSYM][PASTIS_NSYM];
    for (int x = threadIdx.x; x < PASTIS_NSYM * PASTIS_NSYM; x += blockDim.x) {
        int a = x / PASTIS_NSYM, b = x % PASTIS_NSYM;
        s_exp[a][b] = (int)gmat[a * PASTIS_NSYM + a] - (int)gmat[a * PASTIS_NSYM + b];
    }
    __syncthreads();
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_roots) return;
    uint32_t root = roots[r];
    int dig[6], mn[6];
    {
        uint32_t x = root;
        for (int t = k - 1; t >= 0; --t) { dig[t] = (int)(x % PASTIS_NSYM); x /= PASTIS_NSYM; }
    }
    int shift_total = 0;   // sum of per-position minima (unshifted = shifted + shift_total)
    for (int t = 0; t < k; ++t) {
        int v = s_exp[dig[t]][0];
        for (int b = 1; b < PASTIS_NSYM; ++b) v = min(v, s_exp[dig[t]][b]);
        mn[t] = v;
        shift_total += v;
    }
    const int64_t obase = r * (int64_t)(m + 1);
    out_code[obase] = root;
    out_dist[obase] = 0;
    if (m == 0) return;
    // phase 1: counts by shifted distance
    int cnt[SUBK_DLIM], tmp[SUBK_DLIM];
    for (int x = 0; x < SUBK_DLIM; ++x) cnt[x] = 0;
    cnt[0] = 1;
    for (int t = 0; t < k; ++t) {
        for (int x = 0; x < SUBK_DLIM; ++x) tmp[x] = 0;
        for (int b = 0; b < PASTIS_NSYM; ++b) {
            int sh = s_exp[dig[t]][b] - mn[t];
            for (int x = SUBK_DLIM - 1; x >= sh; --x) tmp[x] += cnt[x - sh];
        }
        for (int x = 0; x < SUBK_DLIM; ++x) cnt[x] = tmp[x];
    }
    const int xr = -shift_total;           // shifted distance of the root itself
    int cut = -1, below = 0, run = 0;
    for (int x = 0; x < SUBK_DLIM; ++x) {
        int here = cnt[x] - (x == xr ? 1 : 0);
        if (run + here >= m) { cut = x; below = run; break; }
        run += here;
    }
    if (cut < 0) { atomicExch(err, 1); return; }
    // slot of the first k-mer at each shifted distance (closer ones come first)
    int base[SUBK_DLIM];
    {
        int acc = 0;
        for (int x = 0; x <= cut; ++x) {
            base[x] = acc;
            acc += cnt[x] - (x == xr ? 1 : 0);
        }
    }
    int quota = m - below;
    // phase 2: depth-first walk in code order, pruned at the cut
    int bsel[6], psum[7];
    int depth = 0;
    psum[0] = 0;
    bsel[0] = -1;
    while (depth >= 0) {
        int b = ++bsel[depth];
        if (b >= PASTIS_NSYM) { --depth; continue; }
        int ps = psum[depth] + s_exp[dig[depth]][b] - mn[depth];
        if (ps > cut) continue;
        if (depth + 1 < k) {
            psum[depth + 1] = ps;
            ++depth;
            bsel[depth] = -1;
            continue;
        }
        // a leaf: the k-mer given by bsel[0..k)
        bool is_root = true;
        uint32_t code = 0;
        for (int t = 0; t < k; ++t) {
            is_root &= (bsel[t] == dig[t]);
            code = code * PASTIS_NSYM + (uint32_t)bsel[t];
        }
        if (is_root) continue;
        if (ps == cut) {
            if (quota == 0) continue;
            --quota;
        }
        int slot = base[ps]++;
        out_code[obase + 1 + slot] = code;
        out_dist[obase + 1 + slot] = ps + shift_total;
    }
}

__global__ void k_present_flags(const uint32_t *col_ptr, int64_t ncodes, uint32_t *flags) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncodes) flags[c] = col_ptr[c + 1] > col_ptr[c] ? 1u : 0u;
}

__global__ void k_gather_roots(const uint32_t *flags, const uint32_t *idx, int64_t ncodes, uint32_t *roots) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncodes && flags[c]) roots[idx[c]] = (uint32_t)c;
}

// Expansion of AS: entry (x, t) of A row i and substitute t of its code becomes
// key = substitute code, value = i << 32 | dist << 16 | pos.  Rows are walked in order,
// so equal substitutes keep ascending i after a stable sort by key.
__global__ void k_expand_as(const int64_t *row_ptr, const uint32_t *row_code, const uint16_t *row_pos,
                            int32_t n, const uint32_t *root_index, const uint32_t *sub_code,
                            const int32_t *sub_dist, int m, uint32_t *keys, uint64_t *vals) {
    int64_t nnz = row_ptr[n];
    int64_t tot = nnz * (m + 1);
    for (int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; y < tot;
         y += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = y / (m + 1);
        int t = (int)(y - x * (m + 1));
        // row of x
        int32_t lo = 0, hi = n - 1;
        while (lo < hi) {
            int32_t mid = (lo + hi + 1) >> 1;
            if (row_ptr[mid] <= x) lo = mid; else hi = mid - 1;
        }
        uint32_t ri = root_index[row_code[x]];
        int64_t sidx = (int64_t)ri * (m + 1) + t;
        keys[y] = sub_code[sidx];
        // distances are biased by 1024 so that (dist, pos) orders as one unsigned word
        vals[y] = ((uint64_t)(uint32_t)lo << 32) | ((uint64_t)(uint32_t)(sub_dist[sidx] + 1024) << 16) | row_pos[x];
    }
}

// After the sort by substitute code: the first entry of each (code, seq) run becomes the
// run's minimum (dist, pos) and is flagged to keep.
__global__ void k_reduce_as_runs(const uint32_t *keys, uint64_t *vals, int64_t n, uint32_t *keep) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    uint32_t key = keys[x];
    uint64_t v = vals[x];
    uint32_t seq = (uint32_t)(v >> 32);
    if (x > 0 && keys[x - 1] == key && (uint32_t)(vals[x - 1] >> 32) == seq) { keep[x] = 0; return; }
    uint32_t best = (uint32_t)(v & 0xFFFFFFFFu);   // dist << 16 | pos, both non-negative
    for (int64_t y = x + 1; y < n && keys[y] == key && (uint32_t)(vals[y] >> 32) == seq; ++y) {
        uint32_t w = (uint32_t)(vals[y] & 0xFFFFFFFFu);
        if (w < best) best = w;
    }
    vals[x] = ((uint64_t)seq << 32) | best;
    keep[x] = 1;
}

__global__ void k_compact_as(const uint32_t *keys, const uint64_t *vals, const uint32_t *keep,
                             const uint32_t *off, int64_t n, int32_t *col_seq, uint16_t *col_pos,
                             uint32_t *code_count, uint32_t *rkeys, uint64_t *rvals) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n || !keep[x]) return;
    uint32_t o = off[x];
    uint32_t seq = (uint32_t)(vals[x] >> 32);
    uint16_t pos = (uint16_t)(vals[x] & 0xFFFF);
    col_seq[o] = (int32_t)seq;
    col_pos[o] = pos;
    atomicAdd(&code_count[keys[x]], 1u);
    rkeys[o] = seq;
    rvals[o] = ((uint64_t)keys[x] << 16) | pos;
}

// row_ptr[r] = first index x with keys[x] >= r (keys sorted ascending), r = 0..n
__global__ void k_row_count_u32(const uint32_t *keys, int64_t nnz, int32_t n, int64_t *row_ptr) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)keys[mid] < r) lo = mid + 1; else hi = mid;
    }
    row_ptr[r] = lo;
}

__global__ void k_split_rows_as(const uint64_t *rvals, int64_t nnz, uint32_t *row_code, uint16_t *row_pos) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nnz) return;
    row_code[x] = (uint32_t)(rvals[x] >> 16);
    row_pos[x] = (uint16_t)(rvals[x] & 0xFFFF);
}

int bits_for_u64(uint64_t v) {
    int b = 0;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

pastis_status launch_subkmers(pastis_ctx *ctx, const uint32_t *d_roots, int64_t n_roots, int k, int m,
                              const pastis_params *params, uint32_t *d_code, int32_t *d_dist) {
    int8_t *dmat;
    PASTIS_WS(dmat, ctx, WS_FLAGS, 1024);
    int *err = (int *)(dmat + 768);
    PASTIS_CUDA_TRY(cudaMemcpyAsync(dmat, params->matrix, 576, cudaMemcpyHostToDevice, ctx->stream));
    PASTIS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    if (n_roots > 0) {
        prof_begin(ctx, "subkmers");
        k_subkmers<<<(unsigned)ceil_div64(n_roots, SUBK_THREADS), SUBK_THREADS, 0, ctx->stream>>>(
            d_roots, n_roots, k, m, dmat, d_code, d_dist, err);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    int herr = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return herr ? PASTIS_ERR_INTERNAL : PASTIS_OK;
}

}  // namespace

extern "C" pastis_status pastis_substitute_kmers(pastis_ctx *ctx, const uint32_t *d_roots, int64_t n_roots,
                                                 const pastis_params *params, uint32_t *d_sub_code,
                                                 int32_t *d_sub_dist) {
    if (!ctx || n_roots < 0 || (n_roots > 0 && (!d_roots || !d_sub_code || !d_sub_dist)))
        return PASTIS_ERR_INVALID_ARG;
    pastis_status s = check_params(params);
    if (s != PASTIS_OK) return s;
    return launch_subkmers(ctx, d_roots, n_roots, params->k, params->m_subs, params, d_sub_code, d_sub_dist);
}

// Sets *flag when a[x] != b[x] for some x < n.
template <typename T>
__global__ void k_differs(const T *__restrict__ a, const T *__restrict__ b, int64_t n, uint32_t *flag) {
    bool d = false;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        d |= a[x] != b[x];
    if (__any_sync(0xffffffffu, d) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// Layout of the kept copy of A's rows: the flag word, then row_ptr, row_code, row_pos.
struct as_keep_view {
    uint32_t *flag;
    int64_t *row_ptr;
    uint32_t *row_code;
    uint16_t *row_pos;
};
static size_t as_keep_bytes(int64_t n, int64_t nnz) {
    return 256 + sizeof(int64_t) * (size_t)(n + 1) + sizeof(uint32_t) * (size_t)nnz + sizeof(uint16_t) * (size_t)nnz + 64;
}
static as_keep_view as_keep_layout(void *base, int64_t n, int64_t nnz) {
    as_keep_view v;
    char *p = (char *)base;
    v.flag = (uint32_t *)p;
    v.row_ptr = (int64_t *)(p + 256);
    v.row_code = (uint32_t *)(v.row_ptr + n + 1);
    v.row_pos = (uint16_t *)(v.row_code + nnz);
    return v;
}

// True when the kept AS was built from this A (same rows, compared on the device), k,
// m and matrix.  Synchronises the stream.
static pastis_status as_kept_matches(pastis_ctx *ctx, const pastis_kmat *A, const pastis_params *p, bool *hit) {
    *hit = false;
    if (!ctx->as_valid || ctx->as_k != p->k || ctx->as_m != p->m_subs || ctx->as_n != A->n_rows ||
        ctx->as_nnz_a != A->nnz || memcmp(ctx->as_mat, p->matrix, sizeof(ctx->as_mat)) != 0)
        return PASTIS_OK;
    cudaStream_t st = ctx->stream;
    const as_keep_view v = as_keep_layout(ctx->ws[WS_AS_KEEP], A->n_rows, A->nnz);
    PASTIS_CUDA_TRY(cudaMemsetAsync(v.flag, 0, sizeof(uint32_t), st));
    const int blocks = ctx->sm_count * 8;
    k_differs<int64_t><<<blocks, 256, 0, st>>>(A->row_ptr, v.row_ptr, (int64_t)A->n_rows + 1, v.flag);
    PASTIS_LAUNCHED(ctx);
    if (A->nnz > 0) {
        k_differs<uint32_t><<<blocks, 256, 0, st>>>(A->row_code, v.row_code, A->nnz, v.flag);
        PASTIS_LAUNCHED(ctx);
        k_differs<uint16_t><<<blocks, 256, 0, st>>>(A->row_pos, v.row_pos, A->nnz, v.flag);
        PASTIS_LAUNCHED(ctx);
    }
    uint32_t h = 1;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&h, v.flag, sizeof(h), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    *hit = h == 0;
    return PASTIS_OK;
}

// Keeps a copy of A's rows beside the AS just built, so that a later product over the
// same A (another row block) reuses it.
static pastis_status as_keep(pastis_ctx *ctx, const pastis_kmat *A, const pastis_params *p, const as_matrix *AS) {
    void *base;
    PASTIS_WS(base, ctx, WS_AS_KEEP, as_keep_bytes(A->n_rows, A->nnz));
    const as_keep_view v = as_keep_layout(base, A->n_rows, A->nnz);
    cudaStream_t st = ctx->stream;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(v.row_ptr, A->row_ptr, sizeof(int64_t) * ((size_t)A->n_rows + 1),
                                    cudaMemcpyDeviceToDevice, st));
    if (A->nnz > 0) {
        PASTIS_CUDA_TRY(cudaMemcpyAsync(v.row_code, A->row_code, sizeof(uint32_t) * (size_t)A->nnz,
                                        cudaMemcpyDeviceToDevice, st));
        PASTIS_CUDA_TRY(cudaMemcpyAsync(v.row_pos, A->row_pos, sizeof(uint16_t) * (size_t)A->nnz,
                                        cudaMemcpyDeviceToDevice, st));
    }
    ctx->as_k = p->k;
    ctx->as_m = p->m_subs;
    ctx->as_n = A->n_rows;
    ctx->as_nnz_a = A->nnz;
    memcpy(ctx->as_mat, p->matrix, sizeof(ctx->as_mat));
    ctx->as_kept = *AS;
    ctx->as_valid = 1;
    return PASTIS_OK;
}

// Builds AS (Sec. IV-C), or reuses the one kept from the last call when A, k, m and the
// matrix are unchanged: S depends only on the k-mers present and AS only on A and S, so
// the row blocks of one job share them.
pastis_status build_as_fresh(pastis_ctx *ctx, const pastis_kmat *A, const pastis_params *p, as_matrix *out);

pastis_status build_as(pastis_ctx *ctx, const pastis_kmat *A, const pastis_params *p, as_matrix *out) {
    bool hit = false;
    pastis_status s = as_kept_matches(ctx, A, p, &hit);
    if (s != PASTIS_OK) return s;
    if (hit) {
        *out = ctx->as_kept;
        return PASTIS_OK;
    }
    ctx->as_valid = 0;
    s = build_as_fresh(ctx, A, p, out);
    if (s != PASTIS_OK) return s;
    return as_keep(ctx, A, p, out);
}

pastis_status build_as_fresh(pastis_ctx *ctx, const pastis_kmat *A, const pastis_params *p, as_matrix *out) {
    cudaStream_t st = ctx->stream;
    const int k = p->k, m = p->m_subs;
    const int64_t ncodes = ipow24(k);
    const int32_t n = A->n_rows;
    const int64_t nnzA = A->nnz;
    // distinct codes present in A, and their index
    uint32_t *flags;
    PASTIS_WS(flags, ctx, WS_SUB_ROOTS, sizeof(uint32_t) * (2 * (size_t)ncodes + 2));
    uint32_t *root_index = flags + ncodes + 1;
    k_present_flags<<<(unsigned)ceil_div64(ncodes, 256), 256, 0, st>>>(A->col_ptr, ncodes, flags);
    PASTIS_LAUNCHED(ctx);
    pastis_status s = exclusive_scan_u32(ctx, flags, root_index, ncodes);
    if (s != PASTIS_OK) return s;
    uint32_t h_nroots = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&h_nroots, root_index + ncodes, 4, cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t nroots = h_nroots;
    uint32_t *roots, *sc;
    int32_t *sd;
    PASTIS_WS(roots, ctx, WS_AS_TMP_KEY, sizeof(uint32_t) * (nroots + 1));
    PASTIS_WS(sc, ctx, WS_SUB_CODE, sizeof(uint32_t) * (nroots + 1) * (m + 1));
    PASTIS_WS(sd, ctx, WS_SUB_DIST, sizeof(int32_t) * (nroots + 1) * (m + 1));
    k_gather_roots<<<(unsigned)ceil_div64(ncodes, 256), 256, 0, st>>>(flags, root_index, ncodes, roots);
    PASTIS_LAUNCHED(ctx);
    s = launch_subkmers(ctx, roots, nroots, k, m, p, sc, sd);
    if (s != PASTIS_OK) return s;
    // expand AS
    const int64_t ne = nnzA * (m + 1);
    if (ne > 0xFFFFFFFFll) return PASTIS_ERR_UNSUPPORTED;
    uint32_t *ka, *kb;
    uint64_t *va, *vb;
    PASTIS_WS(ka, ctx, WS_SORT_KEYS_A, sizeof(uint32_t) * (ne + 1));
    PASTIS_WS(kb, ctx, WS_SORT_KEYS_B, sizeof(uint32_t) * (ne + 1));
    PASTIS_WS(va, ctx, WS_SORT_VALS_A, sizeof(uint64_t) * (ne + 1));
    PASTIS_WS(vb, ctx, WS_SORT_VALS_B, sizeof(uint64_t) * (ne + 1));
    if (ne > 0) {
        int blocks = (int)ceil_div64(ne, 256);
        if (blocks > ctx->sm_count * 32) blocks = ctx->sm_count * 32;
        prof_begin(ctx, "as_expand");
        k_expand_as<<<blocks, 256, 0, st>>>(A->row_ptr, A->row_code, A->row_pos, n, root_index, sc, sd, m,
                                           ka, va);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    uint32_t *sk;
    uint64_t *sv;
    s = radix_sort_u32_u64(ctx, ka, va, kb, vb, ne, bits_for_u64((uint64_t)ncodes), &sk, &sv);
    if (s != PASTIS_OK) return s;
    uint32_t *keep;
    PASTIS_WS(keep, ctx, WS_KMER_TMP, sizeof(uint32_t) * (2 * (size_t)ne + 2));
    uint32_t *off = keep + ne + 1;
    if (ne > 0) {
        prof_begin(ctx, "as_reduce");
        k_reduce_as_runs<<<(unsigned)ceil_div64(ne, 256), 256, 0, st>>>(sk, sv, ne, keep);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    s = exclusive_scan_u32(ctx, keep, off, ne);
    if (s != PASTIS_OK) return s;
    uint32_t h_nnz = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&h_nnz, off + ne, 4, cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t nnz = h_nnz;
    out->nnz = nnz;
    PASTIS_WS(out->col_ptr, ctx, WS_AS_COLPTR, sizeof(uint32_t) * (ncodes + 1));
    PASTIS_WS(out->col_seq, ctx, WS_AS_COLSEQ, sizeof(int32_t) * (nnz + 1));
    PASTIS_WS(out->col_pos, ctx, WS_AS_COLPOS, sizeof(uint16_t) * (nnz + 1));
    PASTIS_WS(out->row_ptr, ctx, WS_AS_ROWPTR, sizeof(int64_t) * (n + 1));
    PASTIS_WS(out->row_code, ctx, WS_AS_CODE, sizeof(uint32_t) * (nnz + 1));
    PASTIS_WS(out->row_pos, ctx, WS_AS_POS, sizeof(uint16_t) * (nnz + 1));
    PASTIS_CUDA_TRY(cudaMemsetAsync(out->col_ptr, 0, sizeof(uint32_t) * (ncodes + 1), st));
    uint32_t *rk = (sk == ka) ? kb : ka;
    uint64_t *rv = (sv == va) ? vb : va;
    if (ne > 0) {
        prof_begin(ctx, "as_compact");
        k_compact_as<<<(unsigned)ceil_div64(ne, 256), 256, 0, st>>>(sk, sv, keep, off, ne, out->col_seq,
                                                                   out->col_pos, out->col_ptr, rk, rv);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    s = exclusive_scan_u32(ctx, out->col_ptr, out->col_ptr, ncodes);
    if (s != PASTIS_OK) return s;
    uint32_t *rko;
    uint64_t *rvo;
    s = radix_sort_u32_u64(ctx, rk, rv, sk, sv, nnz, bits_for_u64((uint64_t)(n > 0 ? n - 1 : 0)), &rko, &rvo);
    if (s != PASTIS_OK) return s;
    prof_begin(ctx, "as_rowptr");
    k_row_count_u32<<<(unsigned)ceil_div64((int64_t)n + 1, 256), 256, 0, st>>>(rko, nnz, n, out->row_ptr);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    if (nnz > 0) {
        k_split_rows_as<<<(unsigned)ceil_div64(nnz, 256), 256, 0, st>>>(rvo, nnz, out->row_code, out->row_pos);
        PASTIS_LAUNCHED(ctx);
    }
    return PASTIS_OK;
}
