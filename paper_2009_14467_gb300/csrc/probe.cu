// Integer-pipe throughput probe (no counterpart in the paper): the measured peak that the
// alignment kernels' roofline divides by.
//
// Every thread runs CHAINS dependency chains of one instruction kind for `iters`
// iterations, each iteration advancing every chain UNROLL times.  Chain c takes chain
// c + 1 as its second operand, so no chain is a repeated operation on loop-invariant
// values that a compiler could fold, and the chains still leave CHAINS-way parallelism.
// The grid is exactly `blocks_per_sm` CTAs per SM, all resident at once, and each CTA times its loop with the
// SM clock, so the result is in warp-instructions per SM clock, independent of the clock
// rate:  (CTAs per SM) x (warps per CTA) x (instructions per warp) / (cycles of a CTA).
#include <vector>

#include "internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int CHAINS = 8;
constexpr int UNROLL = 8;

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// One advance of chain x by instruction kind K (y: the next chain, z: a run-time constant).
template <int K>
__device__ __forceinline__ uint32_t op(uint32_t x, uint32_t y, uint32_t z) {
    if constexpr (K == PASTIS_PROBE_VIADDMAX_S16X2) return __viaddmax_s16x2(x, y, z);
    else if constexpr (K == PASTIS_PROBE_VIMAX3_S16X2_RELU) return __vimax3_s16x2_relu(x, y, z);
    else if constexpr (K == PASTIS_PROBE_VADD2) return __vadd2(x, y);
    else if constexpr (K == PASTIS_PROBE_PRMT) return prmt(x, y, z);
    else if constexpr (K == PASTIS_PROBE_IMAD) return mad_lo(x, y, z);
    else if constexpr (K == PASTIS_PROBE_IMAX) return (uint32_t)max((int)x, (int)y);
    else if constexpr (K == PASTIS_PROBE_LOP3) return (x & y) | z;   // consecutive steps fold: counts overstate
    else if constexpr (K == PASTIS_PROBE_MAX3_ADD2) return 0u;   // handled by the caller
    else return x + y;                                        // PASTIS_PROBE_IADD
}

template <int K>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe(uint32_t y, uint32_t z, int iters, uint32_t *sink,
                                                          long long *cycles) {
    uint32_t x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x * 2654435761u + c * y;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) {
                if constexpr (K == PASTIS_PROBE_MAX3_ADD2)   // even chains: 16x2 max3, odd: 16x2 add
                    x[c] = (c & 1) ? __vadd2(x[c], x[(c + 1) % CHAINS])
                                   : __vimax3_s16x2_relu(x[c], x[(c + 1) % CHAINS], z);
                else
                    x[c] = op<K>(x[c], x[(c + 1) % CHAINS], z);
            }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc ^= x[c];
    if (acc == 0x9e3779b9u) sink[threadIdx.x] = acc;          // keeps the chains live
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// The mix of the Smith-Waterman pass-1 recurrence, per 16x2 register (one row of two
// pairs): a sign-extending byte permute of the profile, the diagonal add, E and F as
// add-and-max, H as the three-way max with zero, Ho = H - o, and the two row keys (a
// multiply-add and a maximum for one pair, a masked or and a maximum for the other):
// 10 instructions, 7 of them maxima, permutes or logic, 3 adds.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_sw_mix(uint32_t y, uint32_t z, int iters, uint32_t *sink,
                                                                 long long *cycles) {
    uint32_t Ho[CHAINS], E[CHAINS], kA[CHAINS], kB[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
        Ho[c] = threadIdx.x + c;
        E[c] = y ^ c;
        kA[c] = z + c;
        kB[c] = z ^ c;
    }
    uint32_t f = y, hup = z, hdiag = y ^ z, jt = threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
        jt = jt - 1u;
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) {
            const uint32_t s = prmt(y, z, 0xc480u + c);
            const uint32_t d = __vadd2(hdiag, s);
            E[c] = __viaddmax_s16x2(E[c], z, Ho[c]);
            f = __viaddmax_s16x2(f, z, hup);
            const uint32_t h = __vimax3_s16x2_relu(d, E[c], f);
            hdiag = Ho[c];
            Ho[c] = __vsub2(h, y);
            hup = Ho[c];
            kA[c] = (uint32_t)max((int)kA[c], (int)mad_lo(Ho[c], z, jt));
            kB[c] = (uint32_t)max((int)kB[c], (int)((Ho[c] & 0xFFFF0000u) | jt));
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t acc = f ^ hup;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc ^= Ho[c] ^ E[c] ^ kA[c] ^ kB[c];
    if (acc == 0x9e3779b9u) sink[threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

using probe_fn = void (*)(uint32_t, uint32_t, int, uint32_t *, long long *);

probe_fn probe_kernel(int kind) {
    switch (kind) {
        case PASTIS_PROBE_VIADDMAX_S16X2: return k_probe<PASTIS_PROBE_VIADDMAX_S16X2>;
        case PASTIS_PROBE_VIMAX3_S16X2_RELU: return k_probe<PASTIS_PROBE_VIMAX3_S16X2_RELU>;
        case PASTIS_PROBE_VADD2: return k_probe<PASTIS_PROBE_VADD2>;
        case PASTIS_PROBE_PRMT: return k_probe<PASTIS_PROBE_PRMT>;
        case PASTIS_PROBE_IMAD: return k_probe<PASTIS_PROBE_IMAD>;
        case PASTIS_PROBE_IMAX: return k_probe<PASTIS_PROBE_IMAX>;
        case PASTIS_PROBE_LOP3: return k_probe<PASTIS_PROBE_LOP3>;
        case PASTIS_PROBE_IADD: return k_probe<PASTIS_PROBE_IADD>;
        case PASTIS_PROBE_SW_MIX: return k_probe_sw_mix;
        case PASTIS_PROBE_MAX3_ADD2: return k_probe<PASTIS_PROBE_MAX3_ADD2>;
        default: return nullptr;
    }
}

}  // namespace

extern "C" pastis_status pastis_probe_int_throughput(pastis_ctx *ctx, int32_t kind, int32_t blocks_per_sm,
                                                     int32_t iters, double *h_warp_inst_per_clk_sm) {
    if (!ctx || !h_warp_inst_per_clk_sm || blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1) return PASTIS_ERR_INVALID_ARG;
    probe_fn fn = probe_kernel(kind);
    if (!fn) return PASTIS_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    const int nblk = ctx->sm_count * blocks_per_sm;
    char *buf;
    PASTIS_WS(buf, ctx, WS_FLAGS, sizeof(long long) * (size_t)nblk + sizeof(uint32_t) * PROBE_THREADS + 64);
    long long *cyc = (long long *)buf;
    uint32_t *sink = (uint32_t *)(cyc + nblk);
    // all CTAs must be resident together for the per-CTA cycles to mean a per-SM rate
    int fit = 0;
    PASTIS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, PROBE_THREADS, 0));
    if (fit < blocks_per_sm) return PASTIS_ERR_UNSUPPORTED;
    fn<<<nblk, PROBE_THREADS, 0, st>>>(0x00030001u, 0x00070005u, iters, sink, cyc);
    PASTIS_LAUNCHED(ctx);
    std::vector<long long> h((size_t)nblk);
    PASTIS_CUDA_TRY(cudaMemcpyAsync(h.data(), cyc, sizeof(long long) * nblk, cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    long long worst = 1;
    for (long long c : h) worst = c > worst ? c : worst;
    // instructions per warp in the timed loop: CHAINS x UNROLL per iteration for one kind,
    // 10 x CHAINS for the recurrence mix (its per-iteration column counter not counted)
    const double per_warp = kind == PASTIS_PROBE_SW_MIX ? 10.0 * CHAINS * (double)iters
                                                         : (double)CHAINS * UNROLL * (double)iters;
    const double warps = (double)blocks_per_sm * (PROBE_THREADS / 32);
    *h_warp_inst_per_clk_sm = warps * per_warp / (double)worst;
    return PASTIS_OK;
}
