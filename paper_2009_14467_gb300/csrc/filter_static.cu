// a10 without allocation: the similarity filter of Sec. IV-F / VI-B (the same keep
// rule, edge fields and pair order as pastis_filter_edges) with its scratch in a fixed
// device array instead of a context's workspace.
//
// Three launches: per-tile counts of kept pairs, one block scanning the tile counts,
// then each tile recomputes its flags and scatters its edges at its offset.  A tile is
// 1,024 consecutive pairs; the scratch holds one count and one offset per tile.
#include "internal.cuh"

#include <atomic>
#include <mutex>

namespace {

constexpr int FS_THREADS = 256;
constexpr int FS_PER_THREAD = 4;
constexpr int FS_TILE = FS_THREADS * FS_PER_THREAD;                    // 1,024 pairs
constexpr int64_t FS_MAX_PAIRS = PASTIS_FILTER_STATIC_MAX_PAIRS;
constexpr int FS_MAX_TILES = (int)(FS_MAX_PAIRS / FS_TILE);            // 4,096
static_assert(FS_MAX_PAIRS % FS_TILE == 0, "the pair limit is a whole number of tiles");
constexpr int FS_SCAN_THREADS = 1024;
static_assert(FS_MAX_TILES == FS_SCAN_THREADS * 4, "one scan block covers every tile");

// Scratch layout in 32-bit words:
//   [0]                          error word (an out-of-range pair index sets it)
//   [1]                          total kept pairs (written by the scan)
//   [64, 64 + MAX_TILES)         kept count of each tile
//   [64 + MAX_TILES, + MAX_TILES) exclusive offset of each tile
constexpr int FS_COUNTS = 64;
constexpr int FS_OFFSETS = FS_COUNTS + FS_MAX_TILES;
constexpr int FS_WORDS = FS_OFFSETS + FS_MAX_TILES;                    // 8,256 words = 33,024 bytes
static_assert(FS_WORDS * 4 == PASTIS_FILTER_STATIC_SCRATCH_BYTES, "header states the scratch size");

}  // namespace

// The scratch of every call on a device (calls on one device therefore run one at a time).
static __device__ __align__(256) uint32_t g_filter_scratch[FS_WORDS];

namespace {

// The keep rule of Sec. IV-F: identity and coverage, both inclusive integer tests on
// the shorter sequence (the query on equal lengths).
__device__ __forceinline__ bool fs_keeps(const pastis_aln &a, int lq, int lt, int ani, int cov) {
    if (a.cols == 0) return false;
    const int span = lq <= lt ? (int)a.qe - (int)a.qb : (int)a.te - (int)a.tb;
    const int L = lq <= lt ? lq : lt;
    return 100 * (int)a.ident >= ani * (int)a.cols && 100 * span >= cov * L;
}

__device__ __forceinline__ bool fs_flag(const int64_t *offsets, int32_t n_seqs, const pastis_cand *pairs,
                                        const pastis_aln *alns, int64_t p, int ani, int cov, uint32_t *err) {
    const pastis_cand c = pairs[p];
    if (c.i < 0 || c.j < 0 || c.i >= n_seqs || c.j >= n_seqs) {
        *err = 1u;
        return false;
    }
    const int lq = (int)(offsets[c.i + 1] - offsets[c.i]), lt = (int)(offsets[c.j + 1] - offsets[c.j]);
    return fs_keeps(alns[p], lq, lt, ani, cov);
}

// Block sum of one value per thread (FS_THREADS threads).
__device__ __forceinline__ uint32_t fs_block_sum(uint32_t v, uint32_t *warp_sums) {
    for (int x = 16; x > 0; x >>= 1) v += __shfl_xor_sync(0xffffffffu, v, x);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) warp_sums[w] = v;
    __syncthreads();
    uint32_t s = 0;
    for (int q = 0; q < FS_THREADS / 32; ++q) s += warp_sums[q];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(FS_THREADS)
k_fs_count(const int64_t *offsets, int32_t n_seqs, const pastis_cand *pairs, const pastis_aln *alns, int64_t n,
           int ani, int cov, uint32_t *scratch) {
    __shared__ uint32_t warp_sums[FS_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * FS_TILE;
    uint32_t kept = 0;
    for (int r = 0; r < FS_PER_THREAD; ++r) {
        const int64_t p = base + r * FS_THREADS + threadIdx.x;
        if (p < n && fs_flag(offsets, n_seqs, pairs, alns, p, ani, cov, scratch)) ++kept;
    }
    const uint32_t total = fs_block_sum(kept, warp_sums);
    if (threadIdx.x == 0) scratch[FS_COUNTS + blockIdx.x] = total;
}

// One block: exclusive scan of the n_tiles tile counts, four per thread.
__global__ void __launch_bounds__(FS_SCAN_THREADS) k_fs_scan(int n_tiles, uint32_t *scratch) {
    __shared__ uint32_t warp_sums[FS_SCAN_THREADS / 32];
    const int t0 = threadIdx.x * 4;
    uint32_t c[4], sum = 0;
    for (int q = 0; q < 4; ++q) {
        c[q] = t0 + q < n_tiles ? scratch[FS_COUNTS + t0 + q] : 0u;
        sum += c[q];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = sum;
    for (int x = 1; x < 32; x <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, x);
        if (lane >= x) incl += y;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int q = 0; q < w; ++q) before += warp_sums[q];
    uint32_t run = before + incl - sum;
    for (int q = 0; q < 4; ++q) {
        if (t0 + q < n_tiles) scratch[FS_OFFSETS + t0 + q] = run;
        run += c[q];
    }
    if (threadIdx.x == FS_SCAN_THREADS - 1) scratch[1] = run;    // the last thread ends at the total
}

__global__ void __launch_bounds__(FS_THREADS)
k_fs_scatter(const int64_t *offsets, int32_t n_seqs, const pastis_cand *pairs, const pastis_aln *alns, int64_t n,
             int ani, int cov, uint32_t *scratch, pastis_edge *out) {
    __shared__ uint32_t warp_sums[FS_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * FS_TILE;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t at = scratch[FS_OFFSETS + blockIdx.x];
    // rounds in pair order: round r covers pairs base + r*256 .. base + r*256 + 255
    for (int r = 0; r < FS_PER_THREAD; ++r) {
        const int64_t p = base + r * FS_THREADS + threadIdx.x;
        const bool keep = p < n && fs_flag(offsets, n_seqs, pairs, alns, p, ani, cov, scratch);
        const uint32_t ballot = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) warp_sums[w] = __popc(ballot);
        __syncthreads();
        uint32_t before = 0, round_total = 0;
        for (int q = 0; q < FS_THREADS / 32; ++q) {
            if (q < w) before += warp_sums[q];
            round_total += warp_sums[q];
        }
        __syncthreads();
        if (keep) {
            const pastis_aln a = alns[p];
            pastis_edge e;
            e.i = pairs[p].i;
            e.j = pairs[p].j;
            e.ident = a.ident;
            e.cols = a.cols;
            e.score = a.score;
            e.weight = __fdiv_rn((float)a.ident, (float)a.cols);
            out[at + before + __popc(ballot & ((1u << lane) - 1u))] = e;
        }
        at += round_total;
    }
}

// The scratch address on each device, looked up with that device current.  Only a
// successful lookup is kept: a failed one (say, made while another thread held a
// global-mode stream capture) returns PASTIS_ERR_CUDA for that call and the next call
// on the device tries again.
constexpr int FS_MAX_DEVICES = 64;
struct fs_device {
    std::mutex mu;
    std::atomic<uint32_t *> ptr{nullptr};
};
fs_device g_fs_devices[FS_MAX_DEVICES];

pastis_status fs_scratch(uint32_t **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PASTIS_ERR_CUDA;
    if (dev < 0 || dev >= FS_MAX_DEVICES) return PASTIS_ERR_UNSUPPORTED;
    fs_device &d = g_fs_devices[dev];
    uint32_t *p = d.ptr.load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(d.mu);
        p = d.ptr.load(std::memory_order_relaxed);
        if (!p) {
            void *q = nullptr;
            if (cudaGetSymbolAddress(&q, g_filter_scratch) != cudaSuccess || q == nullptr) {
                (void)cudaGetLastError();            // leave no sticky error for the caller's next call
                return PASTIS_ERR_CUDA;
            }
            p = (uint32_t *)q;
            d.ptr.store(p, std::memory_order_release);
        }
    }
    *out = p;
    return PASTIS_OK;
}

}  // namespace

extern "C" pastis_status pastis_filter_edges_static(void *stream, const int64_t *d_offsets, int32_t n_seqs,
                                                    const pastis_cand *d_pairs, const pastis_aln *d_alns,
                                                    int64_t n_pairs, const pastis_params *params, pastis_edge *d_out,
                                                    int64_t capacity, int64_t *n_out) {
    if (!n_out || n_pairs < 0 || capacity < 0 || n_seqs < 0) return PASTIS_ERR_INVALID_ARG;
    pastis_status s = check_params(params);
    if (s != PASTIS_OK) return s;
    *n_out = 0;
    if (n_pairs > FS_MAX_PAIRS) return PASTIS_ERR_UNSUPPORTED;
    if (n_pairs == 0) return PASTIS_OK;
    if (!d_offsets || !d_pairs || !d_alns) return PASTIS_ERR_INVALID_ARG;
    uint32_t *scratch = nullptr;
    s = fs_scratch(&scratch);
    if (s != PASTIS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int n_tiles = (int)ceil_div64(n_pairs, FS_TILE);
    // Only the error word has to start at zero; counts, offsets and the total are
    // written in full by every call.
    PASTIS_CUDA_TRY(cudaMemsetAsync(scratch, 0, sizeof(uint32_t), st));
    k_fs_count<<<n_tiles, FS_THREADS, 0, st>>>(d_offsets, n_seqs, d_pairs, d_alns, n_pairs, params->ani_min_pct,
                                               params->cov_min_pct, scratch);
    PASTIS_CUDA_TRY(cudaGetLastError());
    k_fs_scan<<<1, FS_SCAN_THREADS, 0, st>>>(n_tiles, scratch);
    PASTIS_CUDA_TRY(cudaGetLastError());
    uint32_t h[2] = {0, 0};                                  // error word, total
    PASTIS_CUDA_TRY(cudaMemcpyAsync(h, scratch, sizeof(h), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h[0]) return PASTIS_ERR_INVALID_ARG;
    *n_out = h[1];
    if (capacity < (int64_t)h[1]) return PASTIS_ERR_CAPACITY;
    if (h[1] == 0) return PASTIS_OK;
    if (!d_out) return PASTIS_ERR_INVALID_ARG;
    k_fs_scatter<<<n_tiles, FS_THREADS, 0, st>>>(d_offsets, n_seqs, d_pairs, d_alns, n_pairs, params->ani_min_pct,
                                                 params->cov_min_pct, scratch, d_out);
    PASTIS_CUDA_TRY(cudaGetLastError());
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    return PASTIS_OK;
}
