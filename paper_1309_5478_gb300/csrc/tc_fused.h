// Parameters of the fused tensor-core GEMM + select kernel (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include <cuda.h>

#include "internal.h"

namespace knn {

// One problem of a batched launch (device memory, 64-byte aligned for the tensor maps).
struct FusedProblem {
    CUtensorMap tmA;           // queries (reduced precision), box 128 rows
    CUtensorMap tmB;           // corpus, box 256 rows
    int64_t M, N;
    int32_t k_bytes, k, km, cap;
    int64_t self_offset;
    const float* cnorm2;
    const float* E;
    const float* thr;
    const float* q_inv_scale;
    const float* c_inv_scale;
    uint64_t* cand;
    int32_t* count;
    uint64_t* bound;
    uint32_t* flags;
    int32_t spec;              // 1: speculative thresholds during the sweep (columns in natural order)
};

// A work item of a batched launch: one 128-row block of one problem.
struct FusedWork {
    int32_t problem;
    int32_t rb;
};

struct FusedParams {
    const void* xq;            // M x k_bytes reduced-precision queries (BF16 or FP8), 128-byte aligned rows
    const void* xc;            // N x k_bytes reduced-precision corpus
    int64_t M, N;
    int32_t k_bytes;           // padded row length in bytes (multiple of 128)
    int32_t k, km, cap;        // answer size, always-kept candidates, list capacity and stride
    const float* cnorm2;       // |c_j|^2 from the FP32 points, padded with NaN to a multiple of 256
    const float* E;            // per-row bound on |approximate - exact| of d'
    const float* thr;          // per-row d' threshold or nullptr
    int32_t thr_bound;         // 1: thr bounds the answer (rows within it are kept complete, fewer than k
                               // allowed: ROW_BOUNDED) instead of guessing it (fewer than k is a miss)
    const float* q_inv_scale;  // FP8: 1 / per-row scale of the queries
    const float* c_inv_scale;  // FP8: same for the corpus (padded like cnorm2)
    int64_t self_offset;       // >= 0: row i excludes column i + self_offset
    const int32_t* self_col;   // or row i excludes column self_col[i] (non-batched launch; else nullptr)
    uint64_t* cand;            // M x cap candidate keys (value, column)
    int32_t* count;            // M
    uint64_t* bound;           // M: every key left out is > bound
    uint32_t* flags;           // M
    int* status;               // device status word (0, or KNN_ETIMEOUT)
    uint64_t* scratch;         // fused_scratch_words(cap_max, grid) words of global scratch
    unsigned long long* inserted;  // optional: keys appended to candidate lists, summed over rows
    int32_t stages;            // shared-memory pipeline depth (fused_stages)
    int32_t cap_max;           // largest list capacity of the launch (sizes shared memory)
    int32_t n_items;           // work items: row blocks of the problem, or entries of `work`
    int32_t spec;              // 1: speculative thresholds during the sweep (non-batched launch only)
    int32_t perm_a;            // corpus tiles are swept in the order ct * perm_a mod (tiles), perm_a coprime
                               // to the tile count (1 = natural order)
    const float* qnorm2;       // |q_i|^2 (needed with spec_d2)
    float spec_d2;             // speculative start threshold in squared distance for every row (+inf: none)
    const FusedProblem* problems;  // batched launch: problem descriptors (else nullptr)
    const FusedWork* work;     // batched launch: work list, largest items first
    long long wait_limit;      // polls of a bounded wait before the kernel gives up (0: 2^26)
    int32_t rr_on;             // 1: two extra warps re-rank finished row blocks during the sweep
                               // (non-batched launch; shared memory sized with rr = true)
    RerankParams rr;           // the re-rank of the whole problem (rows indexed like the lists)
    // Symmetric k-NN graph (non-batched launch, M == N, queries = corpus): row block rb sweeps
    // only the corpus tiles t >= rb / 2 (its own 256-point super-block and later ones). On the
    // tiles after its own super-block the product x_i . x_j also serves row j: keys (d'_ji, i)
    // with squared distance <= sym_t go to row j's inbox. Half the distance product is computed.
    int32_t sym;
    float sym_t;               // squared-distance threshold of the transposed pairs (the probe's start threshold)
    uint64_t* inbox;           // M x cap_in keys of the transposed pairs
    int32_t* inbox_cnt;        // M, zeroed before the launch (may exceed cap_in: the row then lost keys)
    int32_t cap_in;
    const uint32_t* c2max_bits;  // float bits of max |x|^2 over the points (prep statistics)
};

// Largest candidate-list capacity of the fused form (48 keys per lane of a warp), and the
// capacity of the band probe's largest proposal and of the second pass over rows the
// first could not certify.
constexpr int FUSED_CAP_MAX = 1536;
constexpr int FUSED_CAP_WIDE = 1024;

bool fused_available();
// Pipeline stages that fit with lists of capacity cap (and the re-rank warps' buffers when
// rr) for tiles of bn corpus columns (256: one CTA an SM; 128: two CTAs an SM, batched launches
// with lists of at most 512 keys); 0: does not fit.
int fused_stages(int cap, int precision, bool rr = false, int bn = 256);
size_t fused_scratch_words(int cap, int grid);
int fused_cap(int k, int km);
cudaError_t launch_fused(const FusedParams& p, int precision, int grid, cudaStream_t st);
// Batched launch over p.work (p.problems already holds encoded tensor maps).
cudaError_t launch_fused_batched(const FusedParams& p, int precision, int grid, cudaStream_t st, int bn = 256);
// Encodes the two tensor maps of one problem (host).
bool encode_problem_maps(FusedProblem* prob, const void* xq, const void* xc, int precision, int bn = 256);

}  // namespace knn
