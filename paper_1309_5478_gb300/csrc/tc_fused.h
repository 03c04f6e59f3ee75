// Parameters of the fused tensor-core GEMM + select kernel (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace knn {

struct FusedParams {
    const void* xq;            // M x k_bytes reduced-precision queries (BF16 or FP8), 128-byte aligned rows
    const void* xc;            // N x k_bytes reduced-precision corpus
    int64_t M, N;
    int32_t k_bytes;           // padded row length in bytes (multiple of 128)
    int32_t k, km, cap;        // answer size, always-kept candidates, list capacity and stride
    const float* cnorm2;       // |c_j|^2 from the FP32 points, padded with NaN to a multiple of 256
    const float* E;            // per-row bound on |approximate - exact| of d'
    const float* thr;          // per-row d' threshold or nullptr
    const float* q_inv_scale;  // FP8: 1 / per-row scale of the queries
    const float* c_inv_scale;  // FP8: same for the corpus (padded like cnorm2)
    int64_t self_offset;       // >= 0: row i excludes column i + self_offset
    uint64_t* cand;            // M x cap candidate keys (value, column)
    int32_t* count;            // M
    uint64_t* bound;           // M: every key left out is > bound
    uint32_t* flags;           // M
    int* status;               // device status word (0, or KNN_ETIMEOUT)
    uint64_t* scratch;         // fused_scratch_words(cap, grid) words of global scratch
    int32_t stages;            // shared-memory pipeline depth (fused_stages)
};

bool fused_available();
int fused_stages(int cap, int precision);  // 0: does not fit
size_t fused_scratch_words(int cap, int grid);
int fused_cap(int k, int km);
cudaError_t launch_fused(const FusedParams& p, int precision, int grid, cudaStream_t st);

}  // namespace knn
