// Internal declarations shared by the translation units of libpastis (not installed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pastis.h"

#define PASTIS_NSYM 24
#define PASTIS_MAX_M 128
#define PASTIS_MAX_LEN 65535

// Workspace slots of a context: one growable device buffer each.
enum ws_slot {
    WS_FLAGS = 0,     // small device scalars (error words, counters)
    WS_SORT_KEYS_A, WS_SORT_KEYS_B, WS_SORT_VALS_A, WS_SORT_VALS_B, WS_SORT_HIST,
    WS_KMER_TMP,
    WS_SUB_ROOTS, WS_SUB_CODE, WS_SUB_DIST,
    WS_AS_ROWPTR, WS_AS_CODE, WS_AS_POS, WS_AS_COLPTR, WS_AS_COLSEQ, WS_AS_COLPOS,
    WS_AS_TMP_KEY, WS_AS_KEEP,
    WS_SPG_ROWWORK, WS_SPG_ROWOFF, WS_SPG_TMP, WS_SPG_CURSORS, WS_SPG_BIN,
    WS_SPG_RESULT,
    WS_ALN_SCRATCH, WS_ALN_PASS1, WS_ALN_ORDER, WS_ALN_BOUND, WS_ALN_BOFF,
    WS_FILT_FLAGS, WS_FILT_SCAN, WS_CC,
    WS_MLP,
    WS_TUNE,
    WS_COUNT
};

// Pass-1 stripe layout per query-length bin (set by pastis_sw_layout_set or the tuner).
struct sw_layout { uint8_t extra[PASTIS_SW_BINS]; };
__host__ __device__ static inline int sw_bin(int m) {
    const int b = (m - 1) / PASTIS_SW_BIN_WIDTH;
    return b < 0 ? 0 : (b >= PASTIS_SW_BINS ? PASTIS_SW_BINS - 1 : b);
}

// The AS matrix of A under S (Sec. IV-C) in both views, built inside the overlap
// product; every array lives in the context's workspace.
struct as_matrix {
    int64_t nnz;
    int64_t *row_ptr;
    uint32_t *row_code;
    uint16_t *row_pos;
    uint32_t *col_ptr;   // dense over 24^k codes
    int32_t *col_seq;
    uint16_t *col_pos;
};

// Per-kernel CUDA-event timing (enabled by pastis_ctx_profile).
struct prof_rec {
    const char *name;
    cudaEvent_t ev0, ev1;
};
#define PASTIS_PROF_MAX 8192
#define PASTIS_PROF_NAMES 64

struct pastis_ctx {
    int device;
    cudaStream_t stream;
    void *ws[WS_COUNT];
    size_t ws_bytes[WS_COUNT];
    int64_t launches;
    int sm_count;
    size_t smem_optin;
    // kept result of the last overlap product (two-phase size protocol)
    int64_t spg_n;
    const void *spg_key_a, *spg_key_b;
    int64_t spg_key_nnz;
    int32_t spg_key_m, spg_key_min, spg_key_k, spg_key_r0, spg_key_r1;
    uint32_t spg_key_mat_hash;
    int spg_valid;
    // the AS matrix of the last product with substitutes, kept with what it was built
    // from: k, m, the matrix, and a copy of A's rows (compared on the device)
    int as_valid;
    int32_t as_k, as_m, as_n;
    int64_t as_nnz_a;
    int8_t as_mat[PASTIS_NSYM * PASTIS_NSYM];
    as_matrix as_kept;
    // kept result of the last filter
    int64_t filt_n;
    // profiling: pending event pairs and per-name totals
    int prof_on;
    unsigned long long *d_stats;   // work counters while profiling: see pastis_ctx_stats
    int64_t sort_passes;           // radix-sort element passes while profiling (pastis_ctx_stats [3])
    sw_layout sw_lay;              // pass-1 stripe layout per query-length bin
    int xd_per_warp;               // x-drop extensions per warp in 16-bit lanes (1, 2, 4); 0 = 32-bit lanes
    unsigned long long *d_tune;    // per-bin pass-1 cycles while the tuner runs, else null
    int prof_open;
    int prof_n;
    prof_rec prof[PASTIS_PROF_MAX];
    int prof_names;
    const char *prof_name[PASTIS_PROF_NAMES];
    int64_t prof_count[PASTIS_PROF_NAMES];
    double prof_ms[PASTIS_PROF_NAMES];
};

// Records an event before (begin) and after (end) a kernel when profiling is on.
void prof_begin(pastis_ctx *c, const char *name);
void prof_end(pastis_ctx *c);

// Grows workspace slot s to at least `bytes`; returns nullptr on failure.
void *ws_get(pastis_ctx *c, int s, size_t bytes);

#define PASTIS_CUDA_TRY(expr)                                   \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return PASTIS_ERR_CUDA;          \
    } while (0)

#define PASTIS_LAUNCHED(ctx)                                    \
    do {                                                        \
        (ctx)->launches++;                                      \
        cudaError_t _e = cudaGetLastError();                    \
        if (_e != cudaSuccess) return PASTIS_ERR_CUDA;          \
    } while (0)

#define PASTIS_WS(ptr, ctx, slot, bytes)                        \
    do {                                                        \
        (ptr) = (decltype(ptr))ws_get((ctx), (slot), (bytes));  \
        if (!(ptr)) return PASTIS_ERR_OUT_OF_MEMORY;            \
    } while (0)

static inline int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }

static inline int64_t ipow24(int k) {
    int64_t v = 1;
    for (int t = 0; t < k; ++t) v *= PASTIS_NSYM;
    return v;
}

// Device radix sort (LSD, 8-bit digits, stable) of (uint32 key, uint64 value) pairs.
// Sorts keys[0..n) by bits [0, key_bits); the result lands in *keys_out/*vals_out,
// which point at either the input arrays or the two alternate arrays.
pastis_status radix_sort_u32_u64(pastis_ctx *c, uint32_t *keys, uint64_t *vals,
                                 uint32_t *keys_alt, uint64_t *vals_alt, int64_t n,
                                 int key_bits, uint32_t **keys_out, uint64_t **vals_out);

// Exclusive scan of n uint32 counts into uint32 offsets (n+1 entries, last = total).
pastis_status exclusive_scan_u32(pastis_ctx *c, const uint32_t *in, uint32_t *out, int64_t n);
// Exclusive scan of n int64 values into int64 offsets (n+1 entries).
pastis_status exclusive_scan_i64(pastis_ctx *c, const int64_t *in, int64_t *out, int64_t n);

// Raise the dynamic shared-memory limit of the kernels that size it per call to the
// device's opt-in maximum (the current device; done at context creation).
cudaError_t sw_set_smem_limit(size_t bytes);
cudaError_t spgemm_set_smem_limit(size_t bytes);
cudaError_t radix_set_smem_limit();

// Validates the parameters shared by the calls; returns PASTIS_OK or INVALID_ARG.
pastis_status check_params(const pastis_params *p);
uint32_t params_matrix_hash(const pastis_params *p);
