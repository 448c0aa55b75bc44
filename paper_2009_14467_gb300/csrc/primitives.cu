// Device primitives used by the k-mer and candidate stages: a reduce-then-scan exclusive
// prefix sum and a stable LSD radix sort (8-bit digits) of (uint32 key, uint64 value).
#include "internal.cuh"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T v, T *s_warp, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (SCAN_THREADS / 32) ? s_warp[lane] : T(0);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        if (lane < (SCAN_THREADS / 32)) s_warp[lane] = w;
    }
    __syncthreads();
    T warp_off = warp > 0 ? s_warp[warp - 1] : T(0);
    *total = s_warp[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return warp_off + x - v;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_reduce(const TI *in, int64_t n, TO *sums) {
    __shared__ TO s_warp[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    TO acc = 0;
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; ++it) {
        int64_t x = base + (int64_t)it * SCAN_THREADS + threadIdx.x;
        if (x < n) acc += (TO)in[x];
    }
    TO total;
    block_exclusive_scan<TO>(acc, s_warp, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const TI *in, int64_t n, TO *out,
                                                            const TO *block_off) {
    __shared__ TO s_warp[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    TO v[SCAN_ITEMS];
    TO acc = 0;
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; ++it) {
        int64_t x = base + it;
        v[it] = x < n ? (TO)in[x] : TO(0);
        acc += v[it];
    }
    TO total;
    TO run = block_exclusive_scan<TO>(acc, s_warp, &total) + (block_off ? block_off[blockIdx.x] : TO(0));
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; ++it) {
        int64_t x = base + it;
        if (x < n) out[x] = run;
        run += v[it];
        if (x == n - 1) out[n] = run;
    }
}

template <typename TI, typename TO>
pastis_status scan_rec(pastis_ctx *c, const TI *in, TO *out, int64_t n, TO *tmp, int64_t tmp_len) {
    if (n <= 0) {
        PASTIS_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(TO), c->stream));
        return PASTIS_OK;
    }
    int64_t nb = ceil_div64(n, SCAN_TILE);
    if (nb == 1) {
        k_tile_scan<TI, TO><<<1, SCAN_THREADS, 0, c->stream>>>(in, n, out, nullptr);
        PASTIS_LAUNCHED(c);
        return PASTIS_OK;
    }
    if (tmp_len < 2 * (nb + 1)) return PASTIS_ERR_INTERNAL;
    TO *sums = tmp, *offs = tmp + nb + 1;
    k_tile_reduce<TI, TO><<<(unsigned)nb, SCAN_THREADS, 0, c->stream>>>(in, n, sums);
    PASTIS_LAUNCHED(c);
    pastis_status st = scan_rec<TO, TO>(c, sums, offs, nb, tmp + 2 * (nb + 1), tmp_len - 2 * (nb + 1));
    if (st != PASTIS_OK) return st;
    k_tile_scan<TI, TO><<<(unsigned)nb, SCAN_THREADS, 0, c->stream>>>(in, n, out, offs);
    PASTIS_LAUNCHED(c);
    return PASTIS_OK;
}

int64_t scan_tmp_len(int64_t n) {
    int64_t t = 0;
    while (n > SCAN_TILE) {
        int64_t nb = ceil_div64(n, SCAN_TILE);
        t += 2 * (nb + 1);
        n = nb;
    }
    return t + 2;
}

}  // namespace

// A dedicated workspace slot for scan temporaries would collide when a scan runs inside
// the radix sort; the sort owns WS_SORT_HIST and scans use the slot after it.
#define WS_SCAN_TMP WS_FILT_SCAN

pastis_status exclusive_scan_u32(pastis_ctx *c, const uint32_t *in, uint32_t *out, int64_t n) {
    int64_t tl = scan_tmp_len(n);
    uint32_t *tmp;
    PASTIS_WS(tmp, c, WS_SCAN_TMP, sizeof(uint32_t) * tl);
    return scan_rec<uint32_t, uint32_t>(c, in, out, n, tmp, tl);
}

pastis_status exclusive_scan_i64(pastis_ctx *c, const int64_t *in, int64_t *out, int64_t n) {
    int64_t tl = scan_tmp_len(n);
    int64_t *tmp;
    PASTIS_WS(tmp, c, WS_SCAN_TMP, sizeof(int64_t) * tl);
    return scan_rec<int64_t, int64_t>(c, in, out, n, tmp, tl);
}

// ---------------------------------------------------------------------------------
// Stable LSD radix sort.  Per 8-bit digit: a tile histogram, a scan of the
// (digit, tile) counts in digit-major order, then a scatter in which every warp ranks
// its items in input order with __match_any_sync, so equal digits keep input order.
// ---------------------------------------------------------------------------------
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;   // each warp owns 512 consecutive items

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t *keys, int64_t n, int shift,
                                                        uint32_t *hist, int64_t nb) {
    __shared__ uint32_t s_h[256];
    s_h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int it = 0; it < RS_ITEMS; ++it) {
        int64_t x = base + (int64_t)it * RS_THREADS + threadIdx.x;
        if (x < n) atomicAdd(&s_h[(keys[x] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = s_h[threadIdx.x];
}

// The tile's items are first placed in shared memory in their sorted order (digit, then
// input order), then written out in that order, so consecutive threads write
// consecutive positions of each digit's run in the output.
constexpr size_t RS_SCATTER_SMEM = sizeof(uint64_t) * RS_TILE + sizeof(uint32_t) * RS_TILE +
                                   sizeof(uint32_t) * (2 * RS_WARPS * 256 + 2 * 256 + RS_WARPS);

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t *keys, const uint64_t *vals,
                                                           int64_t n, int shift, const uint32_t *offs,
                                                           int64_t nb, uint32_t *okeys, uint64_t *ovals) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    uint64_t *s_v = reinterpret_cast<uint64_t *>(rs_smem);
    uint32_t *s_k = reinterpret_cast<uint32_t *>(s_v + RS_TILE);
    uint32_t *s_cnt = s_k + RS_TILE;                 // [warp][digit]: counts, then ranks so far
    uint32_t *s_base = s_cnt + RS_WARPS * 256;       // [warp][digit]: start within the digit's run
    uint32_t *s_tstart = s_base + RS_WARPS * 256;    // [digit]: start of the digit's run in the tile
    uint32_t *s_gbase = s_tstart + 256;              // [digit]: its start in the output
    uint32_t *s_wsum = s_gbase + 256;                // [warp]: scan carries
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 256 * RS_WARPS; d += RS_THREADS) s_cnt[d] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    const int64_t base = tile0 + (int64_t)warp * (RS_ITEMS * 32);
    uint32_t k[RS_ITEMS];
    uint64_t v[RS_ITEMS];
    uint32_t dg[RS_ITEMS];
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        int64_t x = base + it * 32 + lane;
        bool ok = x < n;
        k[it] = ok ? keys[x] : 0u;
        v[it] = ok ? vals[x] : 0ull;
        dg[it] = ok ? ((k[it] >> shift) & 255u) : 256u;
    }
    // sweep 1: per-warp digit counts
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        unsigned peers = __match_any_sync(0xffffffffu, dg[it]);
        if (dg[it] < 256u && lane == __ffs(peers) - 1) s_cnt[warp * 256 + dg[it]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: the warps' starts within its run, its total, and the runs' starts in the
    // tile (an exclusive scan over the digits)
    const int d0 = threadIdx.x;                      // RS_THREADS == 256 digits
    uint32_t tot = 0;
    for (int w = 0; w < RS_WARPS; ++w) {
        s_base[w * 256 + d0] = tot;
        tot += s_cnt[w * 256 + d0];
        s_cnt[w * 256 + d0] = 0;
    }
    uint32_t incl = tot;
#pragma unroll
    for (int x = 1; x < 32; x <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, x);
        if (lane >= x) incl += y;
    }
    if (lane == 31) s_wsum[warp] = incl;
    s_gbase[d0] = offs[(int64_t)d0 * nb + blockIdx.x];
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += s_wsum[w];
    s_tstart[d0] = wpre + incl - tot;
    __syncthreads();
    // sweep 2: each item to its place in the tile's sorted order
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        unsigned peers = __match_any_sync(0xffffffffu, dg[it]);
        uint32_t d = dg[it];
        uint32_t before = 0;
        if (d < 256u) before = s_cnt[warp * 256 + d];
        __syncwarp();
        if (d < 256u) {
            if (lane == __ffs(peers) - 1) s_cnt[warp * 256 + d] = before + __popc(peers);
            const uint32_t lp = s_tstart[d] + s_base[warp * 256 + d] + before + __popc(peers & lt_mask);
            s_k[lp] = k[it];
            s_v[lp] = v[it];
        }
        __syncwarp();
    }
    __syncthreads();
    // out in the tile's order: each digit's run lands contiguously
    const int tile_n = (int)min((int64_t)RS_TILE, n - tile0);
    for (int x = threadIdx.x; x < tile_n; x += RS_THREADS) {
        const uint32_t key = s_k[x];
        const uint32_t d = (key >> shift) & 255u;
        const uint32_t pos = s_gbase[d] + ((uint32_t)x - s_tstart[d]);
        okeys[pos] = key;
        ovals[pos] = s_v[x];
    }
}

}  // namespace

pastis_status radix_sort_u32_u64(pastis_ctx *c, uint32_t *keys, uint64_t *vals, uint32_t *keys_alt,
                                 uint64_t *vals_alt, int64_t n, int key_bits, uint32_t **keys_out,
                                 uint64_t **vals_out) {
    *keys_out = keys;
    *vals_out = vals;
    if (n <= 1 || key_bits <= 0) return PASTIS_OK;
    if (n > 0xFFFFFFFFll) return PASTIS_ERR_UNSUPPORTED;
    int64_t nb = ceil_div64(n, RS_TILE);
    uint32_t *hist;
    PASTIS_WS(hist, c, WS_SORT_HIST, sizeof(uint32_t) * (256 * nb + 1) * 2);
    uint32_t *offs = hist + 256 * nb + 1;
    uint32_t *ik = keys, *ok = keys_alt;
    uint64_t *iv = vals, *ov = vals_alt;
    if (c->prof_on) c->sort_passes += n * (int64_t)((key_bits + 7) / 8);
    for (int shift = 0; shift < key_bits; shift += 8) {
        prof_begin(c, "radix_hist");
        k_rs_hist<<<(unsigned)nb, RS_THREADS, 0, c->stream>>>(ik, n, shift, hist, nb);
        PASTIS_LAUNCHED(c);
        prof_end(c);
        pastis_status st = exclusive_scan_u32(c, hist, offs, 256 * nb);
        if (st != PASTIS_OK) return st;
        prof_begin(c, "radix_scatter");
        k_rs_scatter<<<(unsigned)nb, RS_THREADS, RS_SCATTER_SMEM, c->stream>>>(ik, iv, n, shift, offs, nb, ok, ov);
        PASTIS_LAUNCHED(c);
        prof_end(c);
        uint32_t *tk = ik; ik = ok; ok = tk;
        uint64_t *tv = iv; iv = ov; ov = tv;
    }
    *keys_out = ik;
    *vals_out = iv;
    return PASTIS_OK;
}

cudaError_t radix_set_smem_limit() {
    return cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_SCATTER_SMEM);
}
