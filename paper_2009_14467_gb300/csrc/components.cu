// Connected components of the similarity graph (the components-as-families variant of
// Sec. VI-B).  Union-find over all edges at once: each edge finds the roots of its two
// ends and hangs the larger root under the smaller one with a compare-and-swap, retrying
// if the larger one stopped being a root meanwhile.  A parent is never larger than its
// vertex (links and path halving both keep that), so every root is the smallest vertex
// of its tree and the labels do not depend on the order in which the edges ran.
#include <algorithm>

#include "internal.cuh"

namespace {

constexpr int CC_MAX_STEPS = 1 << 24;   // bound on one find walk and on one edge's retries

__device__ __forceinline__ int32_t cc_find(int32_t *parent, int32_t v, int *err) {
    volatile int32_t *vp = parent;
    for (int it = 0; it < CC_MAX_STEPS; ++it) {
        const int32_t p = vp[v];
        if (p == v) return v;
        const int32_t g = vp[p];
        if (g != p) vp[v] = g;          // path halving: g is an ancestor of v, never larger than p
        v = g;
    }
    atomicExch(err, 1);
    return v;
}

__global__ void k_cc_init(int32_t *parent, int32_t n) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) parent[v] = v;
}

__global__ void k_cc_hook(const pastis_edge *edges, int64_t n_edges, int32_t n, int32_t *parent, int *bad,
                          int *err) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_edges;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = edges[x].i, b = edges[x].j;
        if (a < 0 || b < 0 || a >= n || b >= n) { atomicExch(bad, 1); continue; }
        int it = 0;
        for (; it < CC_MAX_STEPS; ++it) {
            const int32_t ra = cc_find(parent, a, err), rb = cc_find(parent, b, err);
            if (ra == rb) break;
            const int32_t lo = ra < rb ? ra : rb, hi = ra < rb ? rb : ra;
            if (atomicCAS(&parent[hi], hi, lo) == hi) break;
        }
        if (it == CC_MAX_STEPS) atomicExch(err, 1);
    }
}

__global__ void k_cc_label(int32_t *parent, int32_t n, int32_t *label, int *err) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        label[v] = cc_find(parent, v, err);
}

}  // namespace

extern "C" pastis_status pastis_components(pastis_ctx *ctx, int32_t n_seqs, const pastis_edge *d_edges,
                                           int64_t n_edges, int32_t *d_labels) {
    if (!ctx || n_seqs < 0 || n_edges < 0) return PASTIS_ERR_INVALID_ARG;
    if (n_seqs == 0) return n_edges == 0 ? PASTIS_OK : PASTIS_ERR_INVALID_ARG;
    if (!d_labels || (n_edges > 0 && !d_edges)) return PASTIS_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    int32_t *parent;
    PASTIS_WS(parent, ctx, WS_CC, sizeof(int32_t) * (size_t)n_seqs + 64);
    int *flags = (int *)(parent + n_seqs);          // [0] bad endpoint, [1] walk ran out
    const int vblocks = (int)std::min<int64_t>(ceil_div64(n_seqs, 256), (int64_t)ctx->sm_count * 8);
    const int eblocks = (int)std::min<int64_t>(std::max<int64_t>(ceil_div64(n_edges, 256), 1), (int64_t)ctx->sm_count * 8);
    PASTIS_CUDA_TRY(cudaMemsetAsync(flags, 0, 2 * sizeof(int), st));
    prof_begin(ctx, "cc_init");
    k_cc_init<<<vblocks, 256, 0, st>>>(parent, n_seqs);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    if (n_edges > 0) {
        prof_begin(ctx, "cc_hook");
        k_cc_hook<<<eblocks, 256, 0, st>>>(d_edges, n_edges, n_seqs, parent, flags, flags + 1);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    prof_begin(ctx, "cc_label");
    k_cc_label<<<vblocks, 256, 0, st>>>(parent, n_seqs, d_labels, flags + 1);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    int h[2] = {0, 0};
    PASTIS_CUDA_TRY(cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h[0]) return PASTIS_ERR_INVALID_ARG;
    if (h[1]) return PASTIS_ERR_INTERNAL;
    return PASTIS_OK;
}
