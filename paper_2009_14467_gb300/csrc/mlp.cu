// Learned prefilter: a 16 -> 256 -> 256 -> 1 MLP over per-pair features that predicts
// whether a candidate pair's alignment will pass the similarity filter (Sec. IV-F), so
// that pairs predicted to fail skip the alignment.  The exact path stays the reference:
// labels come from it, and the kept fraction and edge recall are measured against it.
// (The paper's own lever for fewer alignments is the common-k-mer threshold, Sec. VI,
// which costs 2-3% recall; this is a learned version of the same trade.)
//
// Features (16, float32 -> bf16): log1p(count), the two seed diagonals (pos_i - pos_j)
// scaled by 1/256, their spread, log lengths of i and j, log min/max length, the length
// ratio, the BLOSUM scores of the two seed k-mers and their sum (/ 32), count / shorter
// length, seed-1-present flag, and zeros to 16.
//
// Arithmetic: bf16 weights and activations, float32 accumulation on the tensor cores
// (mma.sync m16n8k16, bf16 inputs, f32 accumulators), float32 master weights and Adam
// moments.  Every product of forward and backward goes through one tiled GEMM kernel;
// bias, ReLU, loss and optimizer steps are small elementwise kernels.
#include <cuda_bf16.h>
#include <math.h>

#include "internal.cuh"

namespace {

constexpr int FEAT = 16, HID = 256;

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// ---------------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------------
__global__ void k_pair_features(const uint8_t *qcodes, const int64_t *qoffsets, const uint8_t *tcodes,
                                const int64_t *toffsets, const pastis_cand *pairs, int64_t n, int k,
                                const int8_t *gmat, __nv_bfloat16 *x) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const pastis_cand c = pairs[p];
    const int64_t qo = qoffsets[c.i], to = toffsets[c.j];
    const float lq = (float)(qoffsets[c.i + 1] - qo), lt = (float)(toffsets[c.j + 1] - to);
    float f[FEAT];
#pragma unroll
    for (int t = 0; t < FEAT; ++t) f[t] = 0.f;
    const bool two = c.qpos[1] != 0xFFFF;
    const float d0 = (float)c.qpos[0] - (float)c.tpos[0];
    const float d1 = two ? (float)c.qpos[1] - (float)c.tpos[1] : d0;
    float s0 = 0.f, s1 = 0.f;
    for (int t = 0; t < k; ++t) {
        s0 += gmat[qcodes[qo + c.qpos[0] + t] * PASTIS_NSYM + tcodes[to + c.tpos[0] + t]];
        if (two) s1 += gmat[qcodes[qo + c.qpos[1] + t] * PASTIS_NSYM + tcodes[to + c.tpos[1] + t]];
    }
    const float mn = fminf(lq, lt), mx = fmaxf(lq, lt);
    f[0] = log1pf((float)c.count);
    f[1] = d0 / 256.f;
    f[2] = d1 / 256.f;
    f[3] = fabsf(d0 - d1) / 256.f;
    f[4] = logf(lq + 1.f);
    f[5] = logf(lt + 1.f);
    f[6] = logf(mn + 1.f);
    f[7] = logf(mx + 1.f);
    f[8] = mn / fmaxf(mx, 1.f);
    f[9] = s0 / 32.f;
    f[10] = s1 / 32.f;
    f[11] = (s0 + s1) / 32.f;
    f[12] = (float)c.count / fmaxf(mn, 1.f);
    f[13] = two ? 1.f : 0.f;
#pragma unroll
    for (int t = 0; t < FEAT; ++t) x[p * FEAT + t] = __float2bfloat16(f[t]);
}

// ---------------------------------------------------------------------------------
// GEMM: C[M x N] = op(A)[M x K] * op(B)[K x N] (+ epilogue), bf16 in, f32 accumulate.
// A is row-major M x K (TA = false) or K x M (TA = true); B is row-major K x N (TB =
// false) or N x K (TB = true).  Block tile 64 x 64, 4 warps, each warp 16 rows x 64
// columns = 8 mma tiles of 16 x 8, K in steps of 16 staged through shared memory.
// Epilogue: EP_F32 stores f32 (optionally accumulating), EP_BIAS_RELU stores
// bf16(relu(acc + bias[n])), EP_BIAS stores f32 acc + bias[n].
// ---------------------------------------------------------------------------------
enum { EP_F32 = 0, EP_F32_ACC = 1, EP_BIAS_RELU = 2, EP_BIAS = 3 };

template <bool TA, bool TB, int EP>
__global__ void __launch_bounds__(128) k_gemm_bf16(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B,
                                                   int M, int N, int K, const float *__restrict__ bias, float *Cf,
                                                   __nv_bfloat16 *Cb) {
    __shared__ __nv_bfloat16 sA[64][16 + 8];      // [m][k], padded
    __shared__ __nv_bfloat16 sB[64][16 + 8];      // [n][k], padded (B stored transposed)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[8][4];
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[t][q] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int x = threadIdx.x; x < 64 * 16; x += 128) {
            const int r = x / 16, kk = x % 16;
            const int m = m0 + r, kg = k0 + kk;
            __nv_bfloat16 va = __float2bfloat16(0.f);
            if (m < M && kg < K) va = TA ? A[(int64_t)kg * M + m] : A[(int64_t)m * K + kg];
            sA[r][kk] = va;
            const int nn = n0 + r;
            __nv_bfloat16 vb = __float2bfloat16(0.f);
            if (nn < N && kg < K) vb = TB ? B[(int64_t)nn * K + kg] : B[(int64_t)kg * N + nn];
            sB[r][kk] = vb;
        }
        __syncthreads();
        // A fragment: rows warp*16 + gid (+8), cols tig*2 (+1) and +8
        const int ar = warp * 16 + gid;
        uint32_t a0 = *reinterpret_cast<const uint32_t *>(&sA[ar][tig * 2]);
        uint32_t a1 = *reinterpret_cast<const uint32_t *>(&sA[ar + 8][tig * 2]);
        uint32_t a2 = *reinterpret_cast<const uint32_t *>(&sA[ar][tig * 2 + 8]);
        uint32_t a3 = *reinterpret_cast<const uint32_t *>(&sA[ar + 8][tig * 2 + 8]);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            // B fragment: k rows tig*2 (+1) and +8, column t*8 + gid
            const int bc = t * 8 + gid;
            uint32_t b0 = *reinterpret_cast<const uint32_t *>(&sB[bc][tig * 2]);
            uint32_t b1 = *reinterpret_cast<const uint32_t *>(&sB[bc][tig * 2 + 8]);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
        __syncthreads();
    }
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int m = m0 + warp * 16 + gid + (q >= 2 ? 8 : 0);
            const int nn = n0 + t * 8 + tig * 2 + (q & 1);
            if (m >= M || nn >= N) continue;
            const float v = acc[t][q];
            const int64_t o = (int64_t)m * N + nn;
            if (EP == EP_F32) Cf[o] = v;
            else if (EP == EP_F32_ACC) Cf[o] += v;
            else if (EP == EP_BIAS_RELU) Cb[o] = __float2bfloat16(fmaxf(v + bias[nn], 0.f));
            else Cf[o] = v + bias[nn];
        }
}

// logits z[r] = h2[r, :] . w3 + b3 (one warp per row)
__global__ void k_head(const __nv_bfloat16 *h2, const __nv_bfloat16 *w3, const float *b3, int64_t n, float *z) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    float s = 0.f;
    for (int c = lane; c < HID; c += 32) s += bf(h2[r * HID + c]) * bf(w3[c]);
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) z[r] = s + b3[0];
}

// Per row: the weighted logistic loss term, dz = w * (sigmoid(z) - y) / n and the
// gradient at layer 2's pre-activation, dh2 = dz * w3 where the activation is positive.
// Reductions over rows happen in the fixed-order kernels below (no float atomics), so a
// training step is deterministic.
__global__ void k_loss_rows(const float *z, const float *y, int64_t n, float pos_weight, const __nv_bfloat16 *h2,
                            const __nv_bfloat16 *w3, float *dz, float *lrow, __nv_bfloat16 *dh2) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float zz = z[r], yy = y[r];
    const float w = yy > 0.5f ? pos_weight : 1.f;
    const float sg = 1.f / (1.f + __expf(-zz));
    const float d = w * (sg - yy) / (float)n;
    if (lane == 0) {
        dz[r] = d;
        const float sp = zz > 0.f ? zz + log1pf(__expf(-zz)) : log1pf(__expf(zz));
        lrow[r] = w * (sp - yy * zz) / (float)n;
    }
    for (int c = lane; c < HID; c += 32) {
        const float hv = bf(h2[r * HID + c]);
        dh2[r * HID + c] = __float2bfloat16(hv > 0.f ? d * bf(w3[c]) : 0.f);
    }
}

// g_w3[c] = sum_r h2[r, c] * dz[r], one thread per column, rows in order
__global__ void k_head_wgrad(const __nv_bfloat16 *h2, const float *dz, int64_t n, float *g_w3) {
    const int c = threadIdx.x;
    float s = 0.f;
    for (int64_t r = 0; r < n; ++r) s += bf(h2[r * HID + c]) * dz[r];
    g_w3[c] = s;
}

// two fixed-order sums over n floats (one block of 256 threads): out0 = sum a, out1 = sum b
__global__ void k_pair_sums(const float *a, const float *b, int64_t n, float *out0, float *out1) {
    __shared__ float sa[256], sb[256];
    float x = 0.f, w = 0.f;
    for (int64_t r = threadIdx.x; r < n; r += 256) { x += a[r]; w += b[r]; }
    sa[threadIdx.x] = x;
    sb[threadIdx.x] = w;
    __syncthreads();
    for (int d = 128; d > 0; d >>= 1) {
        if (threadIdx.x < d) { sa[threadIdx.x] += sa[threadIdx.x + d]; sb[threadIdx.x] += sb[threadIdx.x + d]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { *out0 = sa[0]; if (out1) *out1 = sb[0]; }
}

// dact = bf16(dpre where the activation is positive, else 0)
__global__ void k_relu_back(const float *dpre, const __nv_bfloat16 *act, int64_t total, __nv_bfloat16 *dact) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x < total) dact[x] = __float2bfloat16(bf(act[x]) > 0.f ? dpre[x] : 0.f);
}

// g_b[c] = sum_r (masked) values of column c, rows in order (f32 input or bf16 input)
__global__ void k_colsum_masked_f32(const float *dpre, const __nv_bfloat16 *act, int64_t n, float *g_b) {
    const int c = threadIdx.x;
    float s = 0.f;
    for (int64_t r = 0; r < n; ++r) s += bf(act[r * HID + c]) > 0.f ? dpre[r * HID + c] : 0.f;
    g_b[c] = s;
}

__global__ void k_colsum_bf16(const __nv_bfloat16 *d, int64_t n, float *g_b) {
    const int c = threadIdx.x;
    float s = 0.f;
    for (int64_t r = 0; r < n; ++r) s += bf(d[r * HID + c]);
    g_b[c] = s;
}

// Adam on float32 masters; refreshes the bf16 copies
__global__ void k_adam(float *w, float *m1, float *m2, const float *g, __nv_bfloat16 *wb, int64_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const float gg = g[x];
    const float a = b1 * m1[x] + (1.f - b1) * gg;
    const float b = b2 * m2[x] + (1.f - b2) * gg * gg;
    m1[x] = a;
    m2[x] = b;
    const float v = w[x] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    w[x] = v;
    if (wb) wb[x] = __float2bfloat16(v);
}

__global__ void k_select(const pastis_cand *pairs, const float *z, int64_t n, float thr, uint32_t *flags) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) flags[p] = z[p] >= thr ? 1u : 0u;
}

__global__ void k_select_scatter(const pastis_cand *pairs, const uint32_t *flags, const uint32_t *off, int64_t n,
                                 pastis_cand *out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n && flags[p]) out[off[p]] = pairs[p];
}

template <bool TA, bool TB, int EP>
pastis_status gemm(pastis_ctx *ctx, const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K,
                   const float *bias, float *Cf, __nv_bfloat16 *Cb) {
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    prof_begin(ctx, "mlp_gemm");
    k_gemm_bf16<TA, TB, EP><<<grid, 128, 0, ctx->stream>>>(A, B, M, N, K, bias, Cf, Cb);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    return PASTIS_OK;
}

}  // namespace

static pastis_status features_qt(pastis_ctx *ctx, const uint8_t *d_qcodes, const int64_t *d_qoffsets,
                                 const uint8_t *d_tcodes, const int64_t *d_toffsets, const pastis_cand *d_pairs,
                                 int64_t n_pairs, const pastis_params *params, void *d_x) {
    if (!ctx || n_pairs < 0) return PASTIS_ERR_INVALID_ARG;
    pastis_status s = check_params(params);
    if (s != PASTIS_OK) return s;
    if (n_pairs == 0) return PASTIS_OK;
    if (!d_qcodes || !d_qoffsets || !d_tcodes || !d_toffsets || !d_pairs || !d_x) return PASTIS_ERR_INVALID_ARG;
    int8_t *dmat;
    PASTIS_WS(dmat, ctx, WS_FLAGS, 1024);
    PASTIS_CUDA_TRY(cudaMemcpyAsync(dmat, params->matrix, 576, cudaMemcpyHostToDevice, ctx->stream));
    prof_begin(ctx, "mlp_features");
    k_pair_features<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, ctx->stream>>>(
        d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs, n_pairs, params->k, dmat, (__nv_bfloat16 *)d_x);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    return PASTIS_OK;
}

extern "C" pastis_status pastis_pair_features(pastis_ctx *ctx, const uint8_t *d_codes, const int64_t *d_offsets,
                                              const pastis_cand *d_pairs, int64_t n_pairs, const pastis_params *params,
                                              void *d_x) {
    return features_qt(ctx, d_codes, d_offsets, d_codes, d_offsets, d_pairs, n_pairs, params, d_x);
}

extern "C" pastis_status pastis_pair_features_qt(pastis_ctx *ctx, const uint8_t *d_qcodes,
                                                 const int64_t *d_qoffsets, const uint8_t *d_tcodes,
                                                 const int64_t *d_toffsets, const pastis_cand *d_pairs,
                                                 int64_t n_pairs, const pastis_params *params, void *d_x) {
    return features_qt(ctx, d_qcodes, d_qoffsets, d_tcodes, d_toffsets, d_pairs, n_pairs, params, d_x);
}

// Scratch activations for n rows: h1, h2 (bf16 n x 256), z (f32 n), and for training
// dpre (f32 n x 256), dh (bf16 n x 256), dz (f32 n).
static pastis_status mlp_scratch(pastis_ctx *ctx, int64_t n, bool train, __nv_bfloat16 **h1, __nv_bfloat16 **h2,
                                 float **z, float **dpre, __nv_bfloat16 **dh, float **dz) {
    size_t bytes = (size_t)n * HID * 2 * 2 + (size_t)n * 4 + 256;
    if (train) bytes += (size_t)n * HID * 4 + (size_t)n * HID * 2 + (size_t)n * 4 + 256;
    char *b;
    PASTIS_WS(b, ctx, WS_MLP, bytes);
    *h1 = (__nv_bfloat16 *)b; b += (size_t)n * HID * 2;
    *h2 = (__nv_bfloat16 *)b; b += (size_t)n * HID * 2;
    *z = (float *)b; b += ((size_t)n * 4 + 255) & ~(size_t)255;
    if (train) {
        *dpre = (float *)b; b += (size_t)n * HID * 4;
        *dh = (__nv_bfloat16 *)b; b += (size_t)n * HID * 2;
        *dz = (float *)b;
    }
    return PASTIS_OK;
}

static pastis_status mlp_fwd(pastis_ctx *ctx, const pastis_mlp *net, const __nv_bfloat16 *x, int64_t n,
                             __nv_bfloat16 *h1, __nv_bfloat16 *h2, float *z) {
    pastis_status s = gemm<false, false, EP_BIAS_RELU>(ctx, x, (const __nv_bfloat16 *)net->w1b, (int)n, HID, FEAT,
                                                       net->b1, nullptr, h1);
    if (s != PASTIS_OK) return s;
    s = gemm<false, false, EP_BIAS_RELU>(ctx, h1, (const __nv_bfloat16 *)net->w2b, (int)n, HID, HID, net->b2, nullptr, h2);
    if (s != PASTIS_OK) return s;
    prof_begin(ctx, "mlp_head");
    k_head<<<(unsigned)ceil_div64(n * 32, 256), 256, 0, ctx->stream>>>(h2, (const __nv_bfloat16 *)net->w3b, net->b3,
                                                                       n, z);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    return PASTIS_OK;
}

extern "C" pastis_status pastis_mlp_forward(pastis_ctx *ctx, const pastis_mlp *net, const void *d_x, int64_t n,
                                            float *d_logits) {
    if (!ctx || !net || n < 0 || n > (1 << 30)) return PASTIS_ERR_INVALID_ARG;
    if (n == 0) return PASTIS_OK;
    if (!d_x || !d_logits) return PASTIS_ERR_INVALID_ARG;
    const int64_t chunk = 1 << 20;
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t nr = n - r0 < chunk ? n - r0 : chunk;
        __nv_bfloat16 *h1, *h2, *dh;
        float *z, *dpre, *dz;
        pastis_status s = mlp_scratch(ctx, nr, false, &h1, &h2, &z, &dpre, &dh, &dz);
        if (s != PASTIS_OK) return s;
        s = mlp_fwd(ctx, net, (const __nv_bfloat16 *)d_x + r0 * FEAT, nr, h1, h2, d_logits + r0);
        if (s != PASTIS_OK) return s;
    }
    return PASTIS_OK;
}

extern "C" pastis_status pastis_mlp_train_step(pastis_ctx *ctx, pastis_mlp *net, const void *d_x, const float *d_y,
                                               int64_t n, float lr, float pos_weight, float *d_loss) {
    if (!ctx || !net || n <= 0 || n > (1 << 22) || !d_x || !d_y) return PASTIS_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    __nv_bfloat16 *h1, *h2, *dh;
    float *z, *dpre, *dz;
    pastis_status s = mlp_scratch(ctx, n, true, &h1, &h2, &z, &dpre, &dh, &dz);
    if (s != PASTIS_OK) return s;
    const __nv_bfloat16 *x = (const __nv_bfloat16 *)d_x;
    s = mlp_fwd(ctx, net, x, n, h1, h2, z);
    if (s != PASTIS_OK) return s;
    // gradients (zeroed) live after the parameters in the grad buffer
    const int64_t nw1 = FEAT * HID, nw2 = HID * HID;
    float *g = net->grad;
    float *g_w1 = g, *g_b1 = g_w1 + nw1, *g_w2 = g_b1 + HID, *g_b2 = g_w2 + nw2, *g_w3 = g_b2 + HID, *g_b3 = g_w3 + HID;
    const int64_t ntot = nw1 + HID + nw2 + HID + HID + 1;
    PASTIS_CUDA_TRY(cudaMemsetAsync(g, 0, sizeof(float) * ntot, st));
    float *loss = d_loss;   // may be null
    // per-row loss terms and dz share one float buffer of 2n after z
    float *lrow;
    PASTIS_WS(lrow, ctx, WS_FILT_SCAN, sizeof(float) * (size_t)n + 64);
    prof_begin(ctx, "mlp_loss");
    k_loss_rows<<<(unsigned)ceil_div64(n * 32, 256), 256, 0, st>>>(z, d_y, n, pos_weight, h2,
                                                                   (const __nv_bfloat16 *)net->w3b, dz, lrow, dh);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    k_head_wgrad<<<1, HID, 0, st>>>(h2, dz, n, g_w3);
    PASTIS_LAUNCHED(ctx);
    k_pair_sums<<<1, 256, 0, st>>>(dz, lrow, n, g_b3, loss);
    PASTIS_LAUNCHED(ctx);
    // layer 2: g_w2 = h1^T dh2, g_b2 = colsum(dh2), dpre1 = dh2 w2^T
    s = gemm<true, false, EP_F32>(ctx, h1, dh, HID, HID, (int)n, nullptr, g_w2, nullptr);
    if (s != PASTIS_OK) return s;
    k_colsum_bf16<<<1, HID, 0, st>>>(dh, n, g_b2);
    PASTIS_LAUNCHED(ctx);
    s = gemm<false, true, EP_F32>(ctx, dh, (const __nv_bfloat16 *)net->w2b, (int)n, HID, HID, nullptr, dpre, nullptr);
    if (s != PASTIS_OK) return s;
    // back through the ReLU of layer 1 (dh now holds the layer-1 gradient), g_b1
    k_colsum_masked_f32<<<1, HID, 0, st>>>(dpre, h1, n, g_b1);
    PASTIS_LAUNCHED(ctx);
    k_relu_back<<<(unsigned)ceil_div64(n * HID, 256), 256, 0, st>>>(dpre, h1, n * HID, dh);
    PASTIS_LAUNCHED(ctx);
    // layer 1: g_w1 = x^T dh1
    s = gemm<true, false, EP_F32>(ctx, x, dh, FEAT, HID, (int)n, nullptr, g_w1, nullptr);
    if (s != PASTIS_OK) return s;
    // Adam
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)net->step);
    const float c2 = 1.f - powf(b2, (float)net->step);
    struct seg { float *w; __nv_bfloat16 *wb; int64_t off, n; } segs[6] = {
        {net->w1, (__nv_bfloat16 *)net->w1b, 0, nw1}, {net->b1, nullptr, nw1, HID},
        {net->w2, (__nv_bfloat16 *)net->w2b, nw1 + HID, nw2}, {net->b2, nullptr, nw1 + HID + nw2, HID},
        {net->w3, (__nv_bfloat16 *)net->w3b, nw1 + 2 * HID + nw2, HID}, {net->b3, nullptr, nw1 + 3 * HID + nw2, 1}};
    for (int q = 0; q < 6; ++q) {
        prof_begin(ctx, "mlp_adam");
        k_adam<<<(unsigned)ceil_div64(segs[q].n, 256), 256, 0, st>>>(segs[q].w, net->adam_m + segs[q].off,
                                                                     net->adam_v + segs[q].off, g + segs[q].off,
                                                                     segs[q].wb, segs[q].n, lr, b1, b2, 1e-8f, c1, c2);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    return PASTIS_OK;
}

extern "C" pastis_status pastis_prefilter_select(pastis_ctx *ctx, const pastis_cand *d_pairs, const float *d_logits,
                                                 int64_t n_pairs, float threshold, pastis_cand *d_out,
                                                 int64_t capacity, int64_t *n_out) {
    if (!ctx || !n_out || n_pairs < 0 || capacity < 0) return PASTIS_ERR_INVALID_ARG;
    *n_out = 0;
    if (n_pairs == 0) return PASTIS_OK;
    if (!d_pairs || !d_logits) return PASTIS_ERR_INVALID_ARG;
    if (n_pairs > 0xFFFFFFFFll) return PASTIS_ERR_UNSUPPORTED;
    cudaStream_t st = ctx->stream;
    uint32_t *flags;
    PASTIS_WS(flags, ctx, WS_FILT_FLAGS, sizeof(uint32_t) * (2 * (size_t)n_pairs + 2) + 16);
    uint32_t *off = flags + n_pairs + 1;
    k_select<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(d_pairs, d_logits, n_pairs, threshold, flags);
    PASTIS_LAUNCHED(ctx);
    pastis_status s = exclusive_scan_u32(ctx, flags, off, n_pairs);
    if (s != PASTIS_OK) return s;
    uint32_t total = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&total, off + n_pairs, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    *n_out = total;
    if (capacity < (int64_t)total) return PASTIS_ERR_CAPACITY;
    if (total == 0) return PASTIS_OK;
    if (!d_out) return PASTIS_ERR_INVALID_ARG;
    k_select_scatter<<<(unsigned)ceil_div64(n_pairs, 256), 256, 0, st>>>(d_pairs, flags, off, n_pairs, d_out);
    PASTIS_LAUNCHED(ctx);
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    return PASTIS_OK;
}
