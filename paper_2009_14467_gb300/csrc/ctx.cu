// Context, workspace and status strings of libpastis.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "internal.cuh"

void *ws_get(pastis_ctx *c, int s, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c->ws_bytes[s] >= bytes) return c->ws[s];
    if (c->ws[s]) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->ws[s]);
        c->ws[s] = nullptr;
        c->ws_bytes[s] = 0;
    }
    size_t grow = bytes + bytes / 8;            // headroom against repeated regrowth
    grow = (grow + 255) & ~(size_t)255;
    void *p = nullptr;
    if (cudaMalloc(&p, grow) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        grow = bytes;
    }
    c->ws[s] = p;
    c->ws_bytes[s] = grow;
    return p;
}

extern "C" pastis_status pastis_ctx_create(pastis_ctx **ctx, int device, void *stream) {
    if (!ctx) return PASTIS_ERR_INVALID_ARG;
    *ctx = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return PASTIS_ERR_CUDA; }
    if (device < 0 || device >= ndev) return PASTIS_ERR_INVALID_ARG;
    PASTIS_CUDA_TRY(cudaSetDevice(device));
    pastis_ctx *c = (pastis_ctx *)calloc(1, sizeof(pastis_ctx));
    if (!c) return PASTIS_ERR_OUT_OF_MEMORY;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { free(c); return PASTIS_ERR_CUDA; }
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    c->xd_per_warp = PASTIS_XD_DEFAULT_PER_WARP;
    // Kernels with a per-call dynamic shared-memory size get the device's limit once
    // here; a per-call setting could lower it under a launch of another thread.
    if (sw_set_smem_limit(c->smem_optin) != cudaSuccess || spgemm_set_smem_limit(c->smem_optin) != cudaSuccess ||
        radix_set_smem_limit() != cudaSuccess) {
        cudaGetLastError();
        free(c);
        return PASTIS_ERR_CUDA;
    }
    *ctx = c;
    return PASTIS_OK;
}

static void prof_flush(pastis_ctx *c) {
    if (c->prof_n == 0) return;
    cudaStreamSynchronize(c->stream);
    for (int r = 0; r < c->prof_n; ++r) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->prof[r].ev0, c->prof[r].ev1) != cudaSuccess) { cudaGetLastError(); ms = 0.f; }
        int x = 0;
        while (x < c->prof_names && strcmp(c->prof_name[x], c->prof[r].name) != 0) ++x;
        if (x == c->prof_names && x < PASTIS_PROF_NAMES) { c->prof_name[x] = c->prof[r].name; c->prof_count[x] = 0; c->prof_ms[x] = 0; c->prof_names++; }
        if (x < PASTIS_PROF_NAMES) { c->prof_count[x]++; c->prof_ms[x] += ms; }
        cudaEventDestroy(c->prof[r].ev0);
        cudaEventDestroy(c->prof[r].ev1);
    }
    c->prof_n = 0;
}

void prof_begin(pastis_ctx *c, const char *name) {
    if (!c->prof_on) return;
    if (c->prof_open) {                     // an unmatched begin (its launch failed): drop it
        cudaEventDestroy(c->prof[c->prof_n].ev0);
        cudaEventDestroy(c->prof[c->prof_n].ev1);
        c->prof_open = 0;
    }
    if (c->prof_n >= PASTIS_PROF_MAX) prof_flush(c);
    prof_rec &r = c->prof[c->prof_n];
    r.name = name;
    if (cudaEventCreate(&r.ev0) != cudaSuccess) { cudaGetLastError(); return; }
    if (cudaEventCreate(&r.ev1) != cudaSuccess) { cudaGetLastError(); cudaEventDestroy(r.ev0); return; }
    cudaEventRecord(r.ev0, c->stream);
    c->prof_open = 1;
}

void prof_end(pastis_ctx *c) {
    if (!c->prof_on || !c->prof_open) return;
    cudaEventRecord(c->prof[c->prof_n].ev1, c->stream);
    c->prof_n++;
    c->prof_open = 0;
}

extern "C" pastis_status pastis_ctx_profile(pastis_ctx *ctx, int enable) {
    if (!ctx) return PASTIS_ERR_INVALID_ARG;
    prof_flush(ctx);
    if (enable) {
        ctx->prof_names = 0;
        if (!ctx->d_stats && cudaMalloc(&ctx->d_stats, PASTIS_STATS * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            ctx->d_stats = nullptr;
            return PASTIS_ERR_OUT_OF_MEMORY;
        }
        PASTIS_CUDA_TRY(cudaMemsetAsync(ctx->d_stats, 0, PASTIS_STATS * sizeof(unsigned long long), ctx->stream));
        ctx->sort_passes = 0;
    }
    ctx->prof_on = enable ? 1 : 0;
    ctx->prof_open = 0;
    return PASTIS_OK;
}

extern "C" pastis_status pastis_ctx_stats(pastis_ctx *ctx, int64_t *h_out, int32_t n) {
    if (!ctx || !h_out || n < 0) return PASTIS_ERR_INVALID_ARG;
    unsigned long long v[PASTIS_STATS] = {0, 0, 0, 0};
    if (ctx->d_stats) {
        PASTIS_CUDA_TRY(cudaMemcpyAsync(v, ctx->d_stats, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
        PASTIS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    v[3] = (unsigned long long)ctx->sort_passes;
    for (int x = 0; x < n; ++x) h_out[x] = x < PASTIS_STATS ? (int64_t)v[x] : 0;
    return PASTIS_OK;
}

extern "C" int32_t pastis_ctx_profile_read(pastis_ctx *ctx, char *buf, int32_t len) {
    if (!ctx || !buf || len <= 0) return 0;
    prof_flush(ctx);
    int32_t w = 0;
    buf[0] = 0;
    for (int x = 0; x < ctx->prof_names; ++x) {
        int r = snprintf(buf + w, (size_t)(len - w), "%s %lld %.6f\n", ctx->prof_name[x],
                         (long long)ctx->prof_count[x], ctx->prof_ms[x]);
        if (r < 0 || r >= len - w) break;
        w += r;
    }
    return w;
}

extern "C" pastis_status pastis_ctx_destroy(pastis_ctx *ctx) {
    if (!ctx) return PASTIS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    prof_flush(ctx);
    for (int s = 0; s < WS_COUNT; ++s)
        if (ctx->ws[s]) cudaFree(ctx->ws[s]);
    if (ctx->d_stats) cudaFree(ctx->d_stats);
    free(ctx);
    return PASTIS_OK;
}

extern "C" pastis_status pastis_ctx_forget(pastis_ctx *ctx) {
    if (!ctx) return PASTIS_ERR_INVALID_ARG;
    ctx->spg_valid = 0;
    ctx->as_valid = 0;
    return PASTIS_OK;
}

extern "C" int64_t pastis_ctx_workspace_bytes(const pastis_ctx *ctx) {
    if (!ctx) return 0;
    int64_t t = 0;
    for (int s = 0; s < WS_COUNT; ++s) t += (int64_t)ctx->ws_bytes[s];
    return t;
}

extern "C" int64_t pastis_ctx_launch_count(const pastis_ctx *ctx) {
    return ctx ? ctx->launches : 0;
}

extern "C" const char *pastis_status_string(pastis_status s) {
    switch (s) {
        case PASTIS_OK: return "ok";
        case PASTIS_ERR_INVALID_ARG: return "invalid argument";
        case PASTIS_ERR_INVALID_RESIDUE: return "byte outside the residue alphabet";
        case PASTIS_ERR_CAPACITY: return "output buffer too small";
        case PASTIS_ERR_OUT_OF_MEMORY: return "device workspace allocation failed";
        case PASTIS_ERR_CUDA: return "CUDA runtime error";
        case PASTIS_ERR_TIMEOUT: return "bounded device wait expired";
        case PASTIS_ERR_UNSUPPORTED: return "unsupported request";
        case PASTIS_ERR_INTERNAL: return "device consistency check failed";
        default: return "unknown status";
    }
}

pastis_status check_params(const pastis_params *p) {
    if (!p) return PASTIS_ERR_INVALID_ARG;
    if (p->k < 1 || p->k > 6) return PASTIS_ERR_INVALID_ARG;
    if (p->m_subs < 0 || p->m_subs > PASTIS_MAX_M) return PASTIS_ERR_INVALID_ARG;
    if (p->m_subs > ipow24(p->k) - 1) return PASTIS_ERR_INVALID_ARG;
    if (p->min_shared < 1) return PASTIS_ERR_INVALID_ARG;
    if (p->mode != PASTIS_SW && p->mode != PASTIS_XD && p->mode != PASTIS_SW_SCORE && p->mode != PASTIS_SW_FILTERED &&
        p->mode != PASTIS_XD_FILTERED)
        return PASTIS_ERR_INVALID_ARG;
    if (p->xdrop < 0 || p->xdrop > 1000000) return PASTIS_ERR_INVALID_ARG;
    if (p->gap_open < 0 || p->gap_extend < 0 || p->gap_open > 1000 || p->gap_extend > 1000)
        return PASTIS_ERR_INVALID_ARG;
    if (p->ani_min_pct < 0 || p->ani_min_pct > 100 || p->cov_min_pct < 0 || p->cov_min_pct > 100)
        return PASTIS_ERR_INVALID_ARG;
    for (int a = 0; a < PASTIS_NSYM; ++a)
        for (int b = 0; b < PASTIS_NSYM; ++b) {
            int v = p->matrix[a * PASTIS_NSYM + b];
            if (v != p->matrix[b * PASTIS_NSYM + a]) return PASTIS_ERR_INVALID_ARG;
            if (v < -64 || v > 63) return PASTIS_ERR_INVALID_ARG;
        }
    return PASTIS_OK;
}

uint32_t params_matrix_hash(const pastis_params *p) {
    uint32_t h = 2166136261u;      // FNV-1a over the matrix bytes
    for (int x = 0; x < PASTIS_NSYM * PASTIS_NSYM; ++x) {
        h ^= (uint8_t)p->matrix[x];
        h *= 16777619u;
    }
    return h;
}
