// a1-a3: residue encoding, k-mer codes and the sequence x k-mer matrix A.
//
// Sec. V-B: residues are indexed 0..23 in the order ARNDCQEGHILKMFPSTWYVBZX*, and a
// k-mer's id weights the residue i places from the right by 24^i.  Sec. IV-A: A holds
// the start position of k-mer j in sequence i.  One (code, seq, pos) tuple per
// window is radix-sorted by code (stable, so seq and pos stay ascending); the first
// tuple of every (code, seq) run is kept, giving the CSC posting lists (the "tr. A" of
// the paper's dissection); a second stable radix sort by sequence gives the CSR rows
// with codes ascending.
#include "internal.cuh"

namespace {

__constant__ char c_alphabet[PASTIS_NSYM + 1] = "ARNDCQEGHILKMFPSTWYVBZX*";

__global__ void k_encode(const uint8_t *__restrict__ in, int64_t n, uint8_t *__restrict__ out,
                         unsigned long long *bad) {
    __shared__ uint8_t lut[256];
    for (int x = threadIdx.x; x < 256; x += blockDim.x) lut[x] = 0xFF;
    __syncthreads();
    if (threadIdx.x < PASTIS_NSYM) lut[(uint8_t)c_alphabet[threadIdx.x]] = (uint8_t)threadIdx.x;
    __syncthreads();
    const bool vec = ((((uintptr_t)in) | ((uintptr_t)out)) & 15) == 0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (vec) {
        int64_t nv = n >> 4;
        for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
            uint4 w = reinterpret_cast<const uint4 *>(in)[v];
            uint32_t ws[4] = {w.x, w.y, w.z, w.w};
            uint32_t os[4];
            bool okall = true;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t o = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    uint8_t c = lut[(ws[q] >> (8 * b)) & 0xFF];
                    okall &= (c != 0xFF);
                    o |= (uint32_t)c << (8 * b);
                }
                os[q] = o;
            }
            reinterpret_cast<uint4 *>(out)[v] = make_uint4(os[0], os[1], os[2], os[3]);
            if (!okall) {
                for (int b = 0; b < 16; ++b)
                    if (lut[in[v * 16 + b]] == 0xFF) { atomicMin(bad, (unsigned long long)(v * 16 + b)); break; }
            }
        }
        for (int64_t x = (nv << 4) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
            uint8_t c = lut[in[x]];
            out[x] = c;
            if (c == 0xFF) atomicMin(bad, (unsigned long long)x);
        }
    } else {
        for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
            uint8_t c = lut[in[x]];
            out[x] = c;
            if (c == 0xFF) atomicMin(bad, (unsigned long long)x);
        }
    }
}

// One thread per residue position x: the window starting at x, if it fits in its
// sequence, becomes (key = code, value = seq << 16 | pos); otherwise key = invalid,
// which sorts after every code.  Counts the valid windows.
__global__ void k_windows(const uint8_t *__restrict__ codes, const int64_t *__restrict__ offsets,
                          int32_t n, int64_t R, int k, uint32_t invalid, uint32_t *keys,
                          uint64_t *vals, unsigned long long *n_valid, int *bad_code) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = false;
    if (x < R) {
        // sequence of x: the last s with offsets[s] <= x
        int32_t lo = 0, hi = n - 1;
        while (lo < hi) {
            int32_t mid = (lo + hi + 1) >> 1;
            if (offsets[mid] <= x) lo = mid; else hi = mid - 1;
        }
        int64_t p = x - offsets[lo];
        int64_t L = offsets[lo + 1] - offsets[lo];
        uint32_t key = invalid;
        uint64_t val = 0;
        if (p + k <= L) {
            uint32_t c = 0;
            for (int t = 0; t < k; ++t) {
                uint32_t r = codes[x + t];
                if (r >= PASTIS_NSYM) { *bad_code = 1; r = 0; }
                c = c * PASTIS_NSYM + r;
            }
            key = c;
            val = ((uint64_t)(uint32_t)lo << 16) | (uint64_t)p;
            valid = true;
        }
        keys[x] = key;
        vals[x] = val;
    }
    unsigned b = __ballot_sync(0xffffffffu, valid);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_valid, (unsigned long long)__popc(b));
}

// keep[x] = 1 for the first tuple of each (code, seq) run among the valid ones
__global__ void k_first_of_run(const uint32_t *keys, const uint64_t *vals, int64_t nv, uint32_t *keep) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nv) return;
    uint32_t f = 1;
    if (x > 0 && keys[x] == keys[x - 1] && (vals[x] >> 16) == (vals[x - 1] >> 16)) f = 0;
    keep[x] = f;
}

// Compacts the kept tuples into the CSC arrays and prepares the CSR sort input
// (key = seq, value = code << 16 | pos); counts entries per code for col_ptr.
__global__ void k_compact_csc(const uint32_t *keys, const uint64_t *vals, const uint32_t *keep,
                              const uint32_t *keep_off, int64_t nv, int32_t *col_seq, uint16_t *col_pos,
                              uint32_t *code_count, uint32_t *rkeys, uint64_t *rvals) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nv || !keep[x]) return;
    uint32_t o = keep_off[x];
    uint32_t seq = (uint32_t)(vals[x] >> 16);
    uint32_t pos = (uint32_t)(vals[x] & 0xFFFF);
    col_seq[o] = (int32_t)seq;
    col_pos[o] = (uint16_t)pos;
    atomicAdd(&code_count[keys[x]], 1u);
    rkeys[o] = seq;
    rvals[o] = ((uint64_t)keys[x] << 16) | pos;
}

// row_ptr[r] = first index x with keys[x] >= r (keys sorted ascending), r = 0..n
__global__ void k_row_count(const uint32_t *keys, int64_t nnz, int32_t n, int64_t *row_ptr) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)keys[mid] < r) lo = mid + 1; else hi = mid;
    }
    row_ptr[r] = lo;
}

__global__ void k_split_rows(const uint64_t *rvals, int64_t nnz, uint32_t *row_code, uint16_t *row_pos) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nnz) return;
    uint64_t v = rvals[x];
    row_code[x] = (uint32_t)(v >> 16);
    row_pos[x] = (uint16_t)(v & 0xFFFF);
}

__global__ void k_check_offsets(const int64_t *offsets, int32_t n, int *bad) {
    int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int64_t L = offsets[s + 1] - offsets[s];
    if (L < 0 || L > PASTIS_MAX_LEN || (s == 0 && offsets[0] != 0)) *bad = 1;
}

int bits_for(uint64_t v) {   // bits needed to represent values 0..v
    int b = 0;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

}  // namespace

extern "C" pastis_status pastis_encode(pastis_ctx *ctx, const uint8_t *d_ascii, int64_t n_bytes,
                                       uint8_t *d_codes, int64_t *bad_index) {
    if (!ctx || n_bytes < 0 || (n_bytes > 0 && (!d_ascii || !d_codes))) return PASTIS_ERR_INVALID_ARG;
    if (bad_index) *bad_index = -1;
    if (n_bytes == 0) return PASTIS_OK;
    unsigned long long *bad;
    PASTIS_WS(bad, ctx, WS_FLAGS, 64);
    unsigned long long init = ~0ull;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(bad, &init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
    int64_t work = (n_bytes + 15) / 16;
    int blocks = (int)ceil_div64(work, 256);
    int cap = ctx->sm_count * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    prof_begin(ctx, "encode");
    k_encode<<<blocks, 256, 0, ctx->stream>>>(d_ascii, n_bytes, d_codes, bad);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    unsigned long long h = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (h != ~0ull) {
        if (bad_index) *bad_index = (int64_t)h;
        return PASTIS_ERR_INVALID_RESIDUE;
    }
    return PASTIS_OK;
}

extern "C" pastis_status pastis_kmat_sizes(int32_t n, int64_t total_residues, int32_t k,
                                           int64_t *capacity, int64_t *col_ptr_len) {
    if (n < 0 || total_residues < 0 || k < 1 || k > 6) return PASTIS_ERR_INVALID_ARG;
    // every residue starts at most one window, whatever the lengths
    if (capacity) *capacity = total_residues;
    if (col_ptr_len) *col_ptr_len = ipow24(k) + 1;
    return PASTIS_OK;
}

extern "C" pastis_status pastis_build_kmers(pastis_ctx *ctx, const uint8_t *d_codes,
                                            const int64_t *d_offsets, int32_t n, int32_t k,
                                            pastis_kmat *A, int64_t *nnz_out) {
    if (!ctx || !A || !d_offsets || n < 0 || k < 1 || k > 6) return PASTIS_ERR_INVALID_ARG;
    if (A->n_rows != n || A->k != k || !A->row_ptr || !A->col_ptr) return PASTIS_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    const int64_t ncodes = ipow24(k);
    int64_t off_n[2] = {0, 0};
    if (n > 0) {
        PASTIS_CUDA_TRY(cudaMemcpyAsync(&off_n[0], d_offsets, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PASTIS_CUDA_TRY(cudaMemcpyAsync(&off_n[1], d_offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    }
    int *flags;
    PASTIS_WS(flags, ctx, WS_FLAGS, 64);
    unsigned long long *n_valid = (unsigned long long *)(flags + 4);
    PASTIS_CUDA_TRY(cudaMemsetAsync(flags, 0, 64, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t R = off_n[1];
    if (off_n[0] != 0 || R < 0) return PASTIS_ERR_INVALID_ARG;
    if (n > 0) {
        k_check_offsets<<<(unsigned)ceil_div64(n, 256), 256, 0, st>>>(d_offsets, n, flags);
        PASTIS_LAUNCHED(ctx);
    }
    if (R > 0 && !d_codes) return PASTIS_ERR_INVALID_ARG;
    if (R > 0xFFFFFFFFll) return PASTIS_ERR_UNSUPPORTED;

    // col_ptr counts start at zero
    PASTIS_CUDA_TRY(cudaMemsetAsync(A->col_ptr, 0, sizeof(uint32_t) * (ncodes + 1), st));
    PASTIS_CUDA_TRY(cudaMemsetAsync(A->row_ptr, 0, sizeof(int64_t) * (n + 1), st));
    if (R == 0 || n == 0) {
        A->nnz = 0;
        if (nnz_out) *nnz_out = 0;
        PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
        return PASTIS_OK;
    }

    uint32_t *ka, *kb;
    uint64_t *va, *vb;
    PASTIS_WS(ka, ctx, WS_SORT_KEYS_A, sizeof(uint32_t) * R);
    PASTIS_WS(kb, ctx, WS_SORT_KEYS_B, sizeof(uint32_t) * R);
    PASTIS_WS(va, ctx, WS_SORT_VALS_A, sizeof(uint64_t) * R);
    PASTIS_WS(vb, ctx, WS_SORT_VALS_B, sizeof(uint64_t) * R);
    prof_begin(ctx, "kmer_windows");
    k_windows<<<(unsigned)ceil_div64(R, 256), 256, 0, st>>>(d_codes, d_offsets, n, R, k,
                                                          (uint32_t)ncodes, ka, va, n_valid, flags + 1);
    PASTIS_LAUNCHED(ctx);
    prof_end(ctx);
    int hf[2];
    unsigned long long hnv = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&hnv, n_valid, sizeof(hnv), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hf[0]) return PASTIS_ERR_INVALID_ARG;     // offsets not a valid partition
    if (hf[1]) return PASTIS_ERR_INVALID_RESIDUE; // a code >= 24
    const int64_t nv = (int64_t)hnv;
    if (A->capacity < nv || (nv > 0 && (!A->row_code || !A->row_pos || !A->col_seq || !A->col_pos)))
        return PASTIS_ERR_CAPACITY;

    uint32_t *sk;
    uint64_t *sv;
    pastis_status s = radix_sort_u32_u64(ctx, ka, va, kb, vb, R, bits_for((uint64_t)ncodes), &sk, &sv);
    if (s != PASTIS_OK) return s;
    uint32_t *keep;
    PASTIS_WS(keep, ctx, WS_KMER_TMP, sizeof(uint32_t) * (2 * (size_t)nv + 2));
    uint32_t *keep_off = keep + nv + 1;
    if (nv > 0) {
        prof_begin(ctx, "kmer_dedupe");
        k_first_of_run<<<(unsigned)ceil_div64(nv, 256), 256, 0, st>>>(sk, sv, nv, keep);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    s = exclusive_scan_u32(ctx, keep, keep_off, nv);
    if (s != PASTIS_OK) return s;
    uint32_t hnnz = 0;
    PASTIS_CUDA_TRY(cudaMemcpyAsync(&hnnz, keep_off + nv, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t nnz = hnnz;
    // CSR sort input goes to the alternate buffers of the first sort
    uint32_t *rk = (sk == ka) ? kb : ka;
    uint64_t *rv = (sv == va) ? vb : va;
    if (nv > 0) {
        prof_begin(ctx, "kmer_compact");
        k_compact_csc<<<(unsigned)ceil_div64(nv, 256), 256, 0, st>>>(sk, sv, keep, keep_off, nv, A->col_seq,
                                                                   A->col_pos, A->col_ptr, rk, rv);
        PASTIS_LAUNCHED(ctx);
        prof_end(ctx);
    }
    // col_ptr: exclusive scan of per-code counts, in place through the scan's tile order
    s = exclusive_scan_u32(ctx, A->col_ptr, A->col_ptr, ncodes);
    if (s != PASTIS_OK) return s;
    // CSR: stable sort by sequence keeps codes ascending within a row
    uint32_t *rk2 = sk, *rko;
    uint64_t *rv2 = sv, *rvo;
    s = radix_sort_u32_u64(ctx, rk, rv, rk2, rv2, nnz, bits_for((uint64_t)(n - 1)), &rko, &rvo);
    if (s != PASTIS_OK) return s;
    // row pointers: the rows' first indices in the sequence-sorted keys
    k_row_count<<<(unsigned)ceil_div64((int64_t)n + 1, 256), 256, 0, st>>>(rko, nnz, n, A->row_ptr);
    PASTIS_LAUNCHED(ctx);
    if (nnz > 0) {
        k_split_rows<<<(unsigned)ceil_div64(nnz, 256), 256, 0, st>>>(rvo, nnz, A->row_code, A->row_pos);
        PASTIS_LAUNCHED(ctx);
    }
    PASTIS_CUDA_TRY(cudaStreamSynchronize(st));
    A->nnz = nnz;
    if (nnz_out) *nnz_out = nnz;
    ctx->spg_valid = 0;
    return PASTIS_OK;
}
