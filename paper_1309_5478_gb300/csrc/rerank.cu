// Exact re-rank kernels: one warp per row (the row's work is rerank_row of
// rerank_core.cuh: direct-difference FP32 distances of the candidates, early stop past
// the provable k-th distance, FP64 near ties, certificate).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "rerank_core.cuh"
#include "select_core.cuh"

namespace knn {
namespace {

// Block-wide counters: each warp adds its own, then one thread per warp flushes.
__device__ __forceinline__ void block_flush(RerankCounters* counters, unsigned long long (*cnt)[RC_COUNT], int warps) {
    __syncthreads();
    if (threadIdx.x < 32 && static_cast<int>(threadIdx.x) < warps) flush_rerank_counts(counters, cnt[threadIdx.x], false);
}

// One warp per row. With a work counter (next != nullptr) the launch is persistent: every
// warp takes the next row from the counter until none is left, so warps never wait for the
// slowest row of their CTA; without one, warp w of CTA b takes row b * warps + w.
template <bool VEC, int NC, int MINB, int G>
__global__ void __launch_bounds__(256, MINB) rerank_kernel(RerankParams p, int P, unsigned long long* next) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long cnt[8][RC_COUNT];
    const int warp = static_cast<int>(threadIdx.x / 32);
    const int warps = static_cast<int>(blockDim.x / 32);
    const uint32_t lane = lane_id();
    if (lane < RC_COUNT) cnt[warp][lane] = 0ull;
    __syncwarp();
    uint64_t* K = reinterpret_cast<uint64_t*>(smem_raw) + static_cast<size_t>(warp) * (P + TIE_MAX);
    double* T64 = reinterpret_cast<double*>(K + P);
    // a fused kernel that stopped (bounded wait expired) leaves its lists unfinished
    const bool stopped = p.status != nullptr && *p.status != 0;
    int64_t row = static_cast<int64_t>(blockIdx.x) * warps + warp;
    while (!stopped) {
        if (next) {
            unsigned long long r = 0;
            if (lane == 0) r = atomicAdd(next, 1ull);
            row = static_cast<int64_t>(__shfl_sync(0xffffffffu, r, 0));
        }
        if (row >= p.M) break;
        if (!(p.skip_done && (p.row_status[row] & ROW_RERANKED))) {
            const int c = row_keys(p, row);
            if (c >= p.count_min && c <= p.count_max) rerank_row<VEC, NC, G>(p, row, P, K, T64, cnt[warp], lane);
        }
        if (!next) break;
    }
    block_flush(p.counters, cnt, warps);
}

__device__ __forceinline__ int find_seg(const BatchSeg* segs, int32_t nseg, int64_t row) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].row0 <= row) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Every query row of a batch, one warp per row, persistent: warps take the next row (in
// problem order, so a problem's corpus stays in L2 while its rows are re-ranked) from a counter.
__global__ void __launch_bounds__(256, 3)
    rerank_batched_kernel(const BatchDev* __restrict__ probs, const BatchSeg* __restrict__ segs, int32_t nseg,
                          int64_t rows, int P, int32_t count_min, int32_t count_max, RerankCounters* counters,
                          unsigned long long* next) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long cnt[8][RC_COUNT];
    const int warp = static_cast<int>(threadIdx.x / 32);
    const int warps = static_cast<int>(blockDim.x / 32);
    const uint32_t lane = lane_id();
    if (lane < RC_COUNT) cnt[warp][lane] = 0ull;
    __syncwarp();
    for (;;) {
    unsigned long long rr = 0;
    if (lane == 0) rr = atomicAdd(next, 1ull);
    const int64_t row = static_cast<int64_t>(__shfl_sync(0xffffffffu, rr, 0));
    if (row >= rows) break;
    {
        const BatchSeg sg = segs[find_seg(segs, nseg, row)];
        const BatchDev& b = probs[sg.problem];
        RerankParams rp{};
        rp.Q = b.Q;
        rp.C = b.C;
        rp.M = b.M;
        rp.N = b.N;
        rp.d = b.d;
        rp.k = b.k;
        rp.km = b.km;
        rp.cap = b.cap;
        rp.cand = b.cand;
        rp.count = b.count;
        rp.bound = b.bound;
        rp.flags = b.flags;
        rp.E = b.E;
        rp.out_idx = b.out_idx;
        rp.out_dist = b.out_dist;
        rp.row_status = b.row_status;
        rp.uncertified = &b.gq->uncertified;
        const int64_t r = row - sg.row0;
        const int c = list_length(b.count[r], b.flags[r]);
        if (c >= count_min && c <= count_max) {
            uint64_t* K = reinterpret_cast<uint64_t*>(smem_raw) + static_cast<size_t>(warp) * (P + TIE_MAX);
            double* T64 = reinterpret_cast<double*>(K + P);
            const int Pp = pow2_ceil(b.cap > 32 ? b.cap : 32) < P ? pow2_ceil(b.cap > 32 ? b.cap : 32) : P;
            if (b.vec)
                rerank_row<true, 4>(rp, r, Pp, K, T64, cnt[warp], lane);
            else
                rerank_row<false, 4>(rp, r, Pp, K, T64, cnt[warp], lane);
        }
    }
    }
    block_flush(counters, cnt, warps);
}


}  // namespace

namespace {
cudaError_t launch_rerank_batched_range(const BatchDev* probs, const BatchSeg* segs, int32_t nseg, int64_t rows,
                                        int P, int32_t cmin, int32_t cmax, int tier, RerankCounters* counters,
                                        cudaStream_t st) {
    // warps a CTA: as many key buffers as a third of the SM's shared memory holds (at most
    // 8), so that three CTAs share an SM, the most its registers allow at 80 a thread
    // (24 warps for lists of up to 1024 keys, where a fixed 64 KB share gave 21)
    int dev = 0, sms = 0, per_sm = 0, smem_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    const size_t per_warp = static_cast<size_t>(P + TIE_MAX) * 8;
    const size_t share = smem_sm > 3 * 4096 ? static_cast<size_t>(smem_sm) / 3 - 2048 : 64u * 1024u;
    int warps = static_cast<int>(share / per_warp);
    if (warps > 8) warps = 8;
    if (warps < 1) warps = 1;
    const size_t smem = per_warp * warps;
    e = raise_smem_limit(reinterpret_cast<const void*>(rerank_batched_kernel), static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rerank_batched_kernel, warps * 32,
                                                                           smem);
    if (e != cudaSuccess) return e;
    unsigned long long* next = &counters->next_row[tier];
    e = cudaMemsetAsync(next, 0, sizeof(*next), st);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>((rows + warps - 1) / warps, static_cast<int64_t>(std::max(1, per_sm)) * sms);
    rerank_batched_kernel<<<static_cast<unsigned>(blocks), warps * 32, smem, st>>>(probs, segs, nseg, rows, P, cmin,
                                                                                   cmax, counters, next);
    return cudaGetLastError();
}
}  // namespace

// Rows are re-ranked by list length in up to three launches (at most 512, 1024, and the
// largest capacity keys per warp buffer), so that a few long lists do not lower the
// occupancy of the whole batch.
cudaError_t launch_rerank_batched(const BatchDev* probs, const BatchSeg* segs, int32_t nseg, int64_t rows,
                                  int32_t cap_max, RerankCounters* counters, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const int P = pow2_ceil(cap_max > 32 ? cap_max : 32);
    int lo = INT32_MIN;
    int t = 0;
    for (int tier : {512, 1024}) {
        if (P <= tier) break;
        cudaError_t e = launch_rerank_batched_range(probs, segs, nseg, rows, tier, lo, tier, t++, counters, st);
        if (e != cudaSuccess) return e;
        lo = tier + 1;
    }
    return launch_rerank_batched_range(probs, segs, nseg, rows, P, lo, INT32_MAX, t, counters, st);
}

namespace {
using RerankKernel = void (*)(RerankParams, int, unsigned long long*);

// 64 registers a thread (four CTAs of eight warps an SM): the re-rank is bound by the latency
// of its gathers, and more warps in flight beat longer unrolls (measured on GB300: 19.6 ms for
// the 262144-row graph against 20.7 ms at 116 registers and 24.5-26.1 ms with 8-candidate groups).
template <int G>
RerankKernel rerank_variant_g(bool vec) { return vec ? rerank_kernel<true, 4, 4, G> : rerank_kernel<false, 4, 4, G>; }
// lanes per candidate of the distance evaluation by dimension (rerank_group)
RerankKernel rerank_variant(bool vec, int d) {
    switch (rerank_group(d)) {
        case 8: return rerank_variant_g<8>(vec);
        case 16: return rerank_variant_g<16>(vec);
        default: return rerank_variant_g<32>(vec);
    }
}

cudaError_t launch_rerank_range(RerankParams p, int P, int32_t cmin, int32_t cmax, int tier, cudaStream_t st) {
    p.count_min = cmin;
    p.count_max = cmax;
    const size_t per_warp = static_cast<size_t>(P + TIE_MAX) * 8;
    int warps = static_cast<int>((64u * 1024u) / per_warp);
    if (warps > 8) warps = 8;
    if (warps < 1) warps = 1;
    const size_t smem = per_warp * warps;
    const bool vec = (p.d % 4 == 0) && (reinterpret_cast<uintptr_t>(p.Q) % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(p.C) % 16 == 0);
    auto kern = rerank_variant(vec, p.d);
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kern), static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int64_t blocks = (p.M + warps - 1) / warps;
    unsigned long long* next = nullptr;
    if (p.counters) {
        // persistent: as many CTAs as fit at once, rows handed out by a counter
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
        if (e != cudaSuccess) return e;
        next = &p.counters->next_row[tier];
        e = cudaMemsetAsync(next, 0, sizeof(*next), st);
        if (e != cudaSuccess) return e;
        blocks = std::min<int64_t>(blocks, static_cast<int64_t>(std::max(1, per_sm)) * sms);
    }
    kern<<<static_cast<unsigned>(blocks), warps * 32, smem, st>>>(p, P, next);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_rerank(const RerankParams& p, cudaStream_t st) {
    if (p.M <= 0) return cudaSuccess;
    const int keys = p.cap + (p.inbox ? p.cap_in : 0);  // longest list the re-rank may sort
    const int P = pow2_ceil(keys > 32 ? keys : 32);
    int lo = INT32_MIN;
    int t = 0;
    for (int tier : {512, 1024}) {
        if (P <= tier) break;
        cudaError_t e = launch_rerank_range(p, tier, lo, tier, t++, st);
        if (e != cudaSuccess) return e;
        lo = tier + 1;
    }
    return launch_rerank_range(p, P, lo, INT32_MAX, t, st);
}

}  // namespace knn
