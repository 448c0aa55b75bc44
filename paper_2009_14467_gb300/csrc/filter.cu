// a10: the similarity filter and the edges of the similarity graph.
//
// Sec. IV-F: pairs whose alignment identity is below 30% or whose coverage of the
// shorter sequence is below 70% are vetoed; Sec. VI-B: the edge weight is the ANI.
// Both tests are integer comparisons (inclusive); the weight is the correctly rounded
// float32 quotient ident / cols.  Surviving pairs keep their input order (a flag pass,
// an exclusive scan, a scatter).
#include "internal.cuh"

namespace {

__device__ __forceinline__ bool keeps(const pastis_aln &a, int lq, int lt, int ani, int cov) {
    if (a.cols == 0) return false;
    const int span = lq <= lt ? (int)a.qe - (int)a.qb : (int)a.te - (int)a.tb;
    const int L = lq <= lt ? lq : lt;
    return 100 * (int)a.ident >= ani * (int)a.cols && 100 * span >= cov * L;
}

__global__ void k_filter_flags(const int64_t *qoffsets, int32_t n_q, const int64_t *toffsets, int32_t n_t,
                               const pastis_cand *pairs, const pastis_aln *alns, int64_t n, int ani, int cov,
                               uint32_t *flags, int *bad) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const pastis_cand c = pairs[p];
    if (c.i < 0 || c.j < 0 || c.i >= n_q || c.j >= n_t) { *bad = 1; flags[p] = 0; return; }
    const int lq = (int)(qoffsets[c.i + 1] - qoffsets[c.i]), lt = (int)(toffsets[c.j + 1] - toffsets[c.j]);
    flags[p] = keeps(alns[p], lq, lt, ani, cov) ? 1u : 0u;
}

__global__ void k_filter_scatter(const pastis_cand *pairs, const pastis_aln *alns, int64_t n, const uint32_t *flags,
                                 const uint32_t *off, pastis_edge *out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || !flags[p]) return;
    const pastis_aln a = alns[p];
    pastis_edge e;
    e.i = pairs[p].i;
    e.j = pairs[p].j;
    e.ident = a.ident;
    e.cols = a.cols;
    e.score = a.score;
    e.weight = __fdiv_rn((float)a.ident, (float)a.cols);
    out[off[p]] = e;
}

// NS edges (Sec. VI-B): a positive score makes an edge, weighted by score / shorter length.
__global__ void k_ns_flags(const int64_t *offsets, int32_t n_seqs, const pastis_cand *pairs, const pastis_aln *alns,
                           int64_t n, uint32_t *flags, int *bad) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const pastis_cand c = pairs[p];
    if (c.i < 0 || c.j < 0 || c.i >= n_seqs || c.j >= n_seqs) { *bad = 1; flags[p] = 0; return; }
    flags[p] = alns[p].score > 0 ? 1u : 0u;
}

__global__ void k_ns_scatter(const int64_t *offsets, const pastis_cand *pairs, const pastis_aln *alns, int64_t n,
                             const uint32_t *flags, const uint32_t *off, pastis_edge *out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || !flags[p]) return;
    const pastis_cand c = pairs[p];
    const pastis_aln a = alns[p];
    const int64_t lq = offsets[c.i + 1] - offsets[c.i], lt = offsets[c.j + 1] - offsets[c.j];
    pastis_edge e;
    e.i = c.i;
    e.j = c.j;
    e.ident = a.ident;
    e.cols = a.cols;
    e.score = a.score;
    e.weight = __fdiv_rn((float)a.score, (float)(lq < lt ? lq : lt));
    out[off[p]] = e;
}

}  // namespace

extern "C" pastis_status pastis_ns_edges(pastis_ctx *ctx, const int64_t *d_offsets, int32_t n_seqs,
                                         const pastis_cand *d_pairs, const pastis_aln *d_alns, int64_t n_pairs,
                                         pastis_edge *d_out, int64_t capacity, int64_t *n_out) {
    if (!ctx || !n_out || n_pairs < 0 || capacity < 0 || n_seqs < 0) return PASTIS_ERR_INVALID_ARG;
    *n_out = 0;
    if (n_pairs == 0) return PASTIS_OK;
    if (!d_offsets || !d_pairs || !d_alns) return PASTIS_ERR_INVALID_ARG;
    if (n_pairs > 0xFFFFFFFFll) return PASTIS_ERR_UNSUPPORTED;
    cudaStream_t st = ctx->stream;
    uint32_t *flags;
    PASTIS_WS(flags, ctx, WS_FILT_FLAGS, sizeof(uint32_t) * (2 * (size_t)n_pairs + 2) + 16);
    uint32_t *off = flags + n_pairs + 1;
    int *bad = (int *)(off + n_pairs + 1);
    PASTIS_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    const unsigned blocks = (unsigned)ceil_div64(n_pairs, 256);
    prof_begin(ctx, "ns_flags");
    k_ns_flags<<<blocks, 256, 0, st>>>(d_offsets, n_seqs, d_pairs, d_alns, n_pairs, flags, bad);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    pastis_status s = exclusive_scan_u32(ctx, flags, off, n_pairs);
    if (s != PASTIS_OK) return s;
    uint32_t total = 0;
    int hbad = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&total, off + n_pairs, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hbad) return PASTIS_ERR_INVALID_ARG;
    *n_out = total;
    if (capacity < (int64_t)total) return PASTIS_ERR_CAPACITY;
    if (total == 0) return PASTIS_OK;
    if (!d_out) return PASTIS_ERR_INVALID_ARG;
    prof_begin(ctx, "ns_scatter");
    k_ns_scatter<<<blocks, 256, 0, st>>>(d_offsets, d_pairs, d_alns, n_pairs, flags, off, d_out);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    return PASTIS_OK;
}

static pastis_status filter_qt(pastis_ctx *ctx, const int64_t *d_qoffsets, int32_t n_q, const int64_t *d_toffsets,
                               int32_t n_t, const pastis_cand *d_pairs, const pastis_aln *d_alns, int64_t n_pairs,
                               const pastis_params *params, pastis_edge *d_out, int64_t capacity, int64_t *n_out) {
    if (!ctx || !n_out || n_pairs < 0 || capacity < 0 || n_q < 0 || n_t < 0) return PASTIS_ERR_INVALID_ARG;
    pastis_status s = check_params(params);
    if (s != PASTIS_OK) return s;
    *n_out = 0;
    if (n_pairs == 0) return PASTIS_OK;
    if (!d_qoffsets || !d_toffsets || !d_pairs || !d_alns) return PASTIS_ERR_INVALID_ARG;
    if (n_pairs > 0xFFFFFFFFll) return PASTIS_ERR_UNSUPPORTED;
    cudaStream_t st = ctx->stream;
    uint32_t *flags;
    PASTIS_WS(flags, ctx, WS_FILT_FLAGS, sizeof(uint32_t) * (2 * (size_t)n_pairs + 2) + 16);
    uint32_t *off = flags + n_pairs + 1;
    int *bad = (int *)(off + n_pairs + 1);
    PASTIS_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    const unsigned blocks = (unsigned)ceil_div64(n_pairs, 256);
    prof_begin(ctx, "filter_flags");
    k_filter_flags<<<blocks, 256, 0, st>>>(d_qoffsets, n_q, d_toffsets, n_t, d_pairs, d_alns, n_pairs,
                                           params->ani_min_pct, params->cov_min_pct, flags, bad);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    s = exclusive_scan_u32(ctx, flags, off, n_pairs);
    if (s != PASTIS_OK) return s;
    uint32_t total = 0;
    int hbad = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&total, off + n_pairs, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hbad) return PASTIS_ERR_INVALID_ARG;
    *n_out = total;
    if (capacity < (int64_t)total) return PASTIS_ERR_CAPACITY;
    if (total == 0) return PASTIS_OK;
    if (!d_out) return PASTIS_ERR_INVALID_ARG;
    prof_begin(ctx, "filter_scatter");
    k_filter_scatter<<<blocks, 256, 0, st>>>(d_pairs, d_alns, n_pairs, flags, off, d_out);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    return PASTIS_OK;
}

extern "C" pastis_status pastis_filter_edges(pastis_ctx *ctx, const int64_t *d_offsets, int32_t n_seqs,
                                             const pastis_cand *d_pairs, const pastis_aln *d_alns, int64_t n_pairs,
                                             const pastis_params *params, pastis_edge *d_out, int64_t capacity,
                                             int64_t *n_out) {
    return filter_qt(ctx, d_offsets, n_seqs, d_offsets, n_seqs, d_pairs, d_alns, n_pairs, params, d_out, capacity,
                     n_out);
}

extern "C" pastis_status pastis_filter_edges_qt(pastis_ctx *ctx, const int64_t *d_qoffsets, int32_t n_q,
                                                const int64_t *d_toffsets, int32_t n_t, const pastis_cand *d_pairs,
                                                const pastis_aln *d_alns, int64_t n_pairs, const pastis_params *params,
                                                pastis_edge *d_out, int64_t capacity, int64_t *n_out) {
    return filter_qt(ctx, d_qoffsets, n_q, d_toffsets, n_t, d_pairs, d_alns, n_pairs, params, d_out, capacity, n_out);
}
