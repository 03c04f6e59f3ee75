// Exact re-rank of each row's candidate list.
//
// The candidate lists come from the selection (fused or not) on approximate
// ranking values d'_ij = |c_j|^2 - 2 q_i.c_j (Methods, "Distance calculation").
// Here every candidate's squared distance is recomputed in the direct difference
// form sum_t (q_t - c_t)^2, which has no cancellation:
//   - each lane adds its four products of a 16-byte group with FMAs and folds the
//     group sum into a (sum, error) pair with Knuth's TwoSum; the warp reduction adds
//     the pairs with TwoSum as well. The result's relative error is at most about
//     8 units in the last place (2 for the rounded differences, 4 for the group sums,
//     2 for the final roundings), below 2^-20.
//   - the list is sorted by (FP32 distance, index). Neighbours in the sorted list that
//     are within 2^-19 (relative) of each other around the first k positions form
//     near-tie groups; their distances are recomputed in FP64 and the group re-sorted
//     by (FP64 distance, index). FP64 therefore decides only the order of points whose
//     FP32 distances cannot be told apart.
//   - a row whose list was truncated is certified only if the k-th exact distance is
//     below the smallest value any left-out point can have, bound - E (in d' scale).
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "select_core.cuh"

namespace knn {
namespace {

constexpr float TIE_REL = 0x1p-19f;

__device__ __forceinline__ void group_sum(float4 q, float4 c, float& s, float& e) {
    const float d0 = q.x - c.x, d1 = q.y - c.y, d2 = q.z - c.z, d3 = q.w - c.w;
    float g = d0 * d0;
    g = fmaf(d1, d1, g);
    g = fmaf(d2, d2, g);
    g = fmaf(d3, d3, g);
    float t, err;
    two_sum(s, g, t, err);
    s = t;
    e += err;
}

__device__ __forceinline__ float warp_reduce_pair(float s, float e) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float so = __shfl_xor_sync(0xffffffffu, s, o);
        const float eo = __shfl_xor_sync(0xffffffffu, e, o);
        float t, err;
        two_sum(s, so, t, err);
        s = t;
        e = e + eo + err;
    }
    return s + e;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool VEC>
__device__ __forceinline__ float sqdist_fp32(const float* __restrict__ q, const float* __restrict__ c, int d) {
    const uint32_t lane = lane_id();
    float s = 0.f, e = 0.f;
    if (VEC) {
        for (int t = static_cast<int>(lane) * 4; t < d; t += 128) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(q + t));
            const float4 b = __ldg(reinterpret_cast<const float4*>(c + t));
            group_sum(a, b, s, e);
        }
    } else {
        for (int t = static_cast<int>(lane) * 4; t < d; t += 128) {
            float4 a, b;
            a.x = q[t];
            b.x = c[t];
            a.y = t + 1 < d ? q[t + 1] : 0.f;
            b.y = t + 1 < d ? c[t + 1] : 0.f;
            a.z = t + 2 < d ? q[t + 2] : 0.f;
            b.z = t + 2 < d ? c[t + 2] : 0.f;
            a.w = t + 3 < d ? q[t + 3] : 0.f;
            b.w = t + 3 < d ? c[t + 3] : 0.f;
            group_sum(a, b, s, e);
        }
    }
    return warp_reduce_pair(s, e);
}

// Two candidates at once (more loads in flight per lane).
template <bool VEC>
__device__ __forceinline__ void sqdist_fp32_x2(const float* __restrict__ q, const float* __restrict__ c0,
                                               const float* __restrict__ c1, int d, float& r0, float& r1) {
    if (!VEC) {
        r0 = sqdist_fp32<false>(q, c0, d);
        r1 = sqdist_fp32<false>(q, c1, d);
        return;
    }
    const uint32_t lane = lane_id();
    float s0 = 0.f, e0 = 0.f, s1 = 0.f, e1 = 0.f;
    for (int t = static_cast<int>(lane) * 4; t < d; t += 128) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(q + t));
        const float4 b0 = __ldg(reinterpret_cast<const float4*>(c0 + t));
        const float4 b1 = __ldg(reinterpret_cast<const float4*>(c1 + t));
        group_sum(a, b0, s0, e0);
        group_sum(a, b1, s1, e1);
    }
    r0 = warp_reduce_pair(s0, e0);
    r1 = warp_reduce_pair(s1, e1);
}

// Four candidates at once (more loads in flight per lane).
template <bool VEC>
__device__ __forceinline__ void sqdist_fp32_x4(const float* __restrict__ q, const float* const (&c)[4], int d,
                                               float (&r)[4]) {
    if (!VEC) {
#pragma unroll
        for (int i = 0; i < 4; ++i) r[i] = sqdist_fp32<false>(q, c[i], d);
        return;
    }
    const uint32_t lane = lane_id();
    float s[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = static_cast<int>(lane) * 4; t < d; t += 128) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(q + t));
        float4 b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = __ldg(reinterpret_cast<const float4*>(c[i] + t));
#pragma unroll
        for (int i = 0; i < 4; ++i) group_sum(a, b[i], s[i], e[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) r[i] = warp_reduce_pair(s[i], e[i]);
}

__device__ __forceinline__ double sqdist_fp64(const float* __restrict__ q, const float* __restrict__ c, int d) {
    double s = 0.0;
    for (int t = static_cast<int>(lane_id()); t < d; t += 32) {
        const double diff = static_cast<double>(q[t]) - static_cast<double>(c[t]);
        s = fma(diff, diff, s);
    }
    return warp_sum_d(s);
}

__device__ __forceinline__ void flush_counters(RerankCounters* counters, unsigned long long* blk_cnt) {
    __syncthreads();
    if (threadIdx.x == 0 && counters) {
        atomicAdd(&counters->candidates, blk_cnt[0]);
        if (blk_cnt[1]) atomicAdd(&counters->fp64_rows, blk_cnt[1]);
        if (blk_cnt[2]) atomicAdd(&counters->uncertified, blk_cnt[2]);
        if (blk_cnt[3]) atomicAdd(&counters->truncated, blk_cnt[3]);
        if (blk_cnt[4]) atomicAdd(&counters->threshold_miss, blk_cnt[4]);
    }
}

// Members of one near-tie group settled in FP64 at most (a larger group is left unordered
// and its row reported uncertified).
constexpr int TIE_MAX = 128;

// One warp re-ranks row `row` of p; K is the warp's shared-memory array of P keys and T64
// its TIE_MAX doubles for one near-tie group.
template <bool VEC>
__device__ __forceinline__ void rerank_row(const RerankParams& p, int64_t row, int P, uint64_t* K, double* T64,
                                           unsigned long long* blk_cnt, uint32_t lane) {
    {
        const int raw = p.count[row];
        const uint32_t flags = p.flags[row];
        const float* q = p.Q + row * static_cast<int64_t>(p.d);
        const uint64_t* cand = p.cand + row * static_cast<int64_t>(p.cap);
        const int d = p.d;

        // 0. the row's candidate keys into K. A raw list (every key <= bound, in a front and
        //    a back segment) is first reduced to the band of its approximate values, as the
        //    select does: sorted, then the keys <= min(bound, max(key_(k+m), ceiling(v_(k) +
        //    2E))) kept. A row whose bound came from a speculative threshold is truncated
        //    there when that band reaches beyond it.
        int count;
        bool spec_cut = false;
        if (flags & ROW_RAW_LIST) {
            const int n0 = raw & 0xffff, n = n0 + (raw >> 16);
            const int Pn = pow2_ceil(n > 32 ? n : 32) < P ? pow2_ceil(n > 32 ? n : 32) : P;
            for (int i = static_cast<int>(lane); i < Pn; i += 32)
                K[i] = i < n0 ? cand[i] : (i < n ? cand[p.cap - 1 - (i - n0)] : KEY_MAX);
            __syncwarp();
            warp_bitonic_sort_smem(K, Pn);
            const int kk = n < p.k ? n : p.k;
            uint64_t band = KEY_MAX;
            if (n >= p.km && n > 0) {
                band = K[p.km - 1];
                const float window = p.E ? 2.f * p.E[row] : 0.f;
                if (window > 0.f) {
                    const uint64_t wk = key_ceiling(key_val(K[kk - 1]) + window);
                    band = wk > band ? wk : band;
                }
            }
            const uint64_t tau = p.bound[row];
            const uint64_t nt = band < tau ? band : tau;
            int keep = 0;
            for (int i = static_cast<int>(lane); i < n; i += 32) keep += K[i] <= nt ? 1 : 0;
            count = static_cast<int>(__reduce_add_sync(0xffffffffu, static_cast<uint32_t>(keep)));
            spec_cut = (flags & ROW_SPECULATIVE) && (band > tau || n < p.km);
        } else {
            count = raw;
            for (int i = static_cast<int>(lane); i < count; i += 32) K[i] = cand[i];
        }
        __syncwarp();

        // 1. direct-difference FP32 distances, four candidates at a time
        int c = 0;
        for (; c + 3 < count; c += 4) {
            uint32_t j[4];
            const float* cp[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                j[i] = key_idx(K[c + i]);
                cp[i] = p.C + static_cast<int64_t>(j[i]) * d;
            }
            float r[4];
            sqdist_fp32_x4<VEC>(q, cp, d, r);
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) K[c + i] = make_key(r[i], j[i]);
            }
        }
        for (; c + 1 < count; c += 2) {
            const uint32_t j0 = key_idx(K[c]);
            const uint32_t j1 = key_idx(K[c + 1]);
            float r0, r1;
            sqdist_fp32_x2<VEC>(q, p.C + static_cast<int64_t>(j0) * d, p.C + static_cast<int64_t>(j1) * d, d, r0,
                                r1);
            if (lane == 0) {
                K[c] = make_key(r0, j0);
                K[c + 1] = make_key(r1, j1);
            }
        }
        if (c < count) {
            const uint32_t j0 = key_idx(K[c]);
            const float r0 = sqdist_fp32<VEC>(q, p.C + static_cast<int64_t>(j0) * d, d);
            if (lane == 0) K[c] = make_key(r0, j0);
        }
        // sort only the power of two that holds the list (P bounds it)
        const int Pc = pow2_ceil(count > 32 ? count : 32) < P ? pow2_ceil(count > 32 ? count : 32) : P;
        for (int i = count + static_cast<int>(lane); i < Pc; i += 32) K[i] = KEY_MAX;
        __syncwarp();
        warp_bitonic_sort_smem(K, Pc);

        // 2. near ties around the first k positions, settled in FP64 (skipped when the
        //    inputs make FP32 exact: then equal values are true ties, already ordered by index)
        const int k = p.k;
        const int kk = count < k ? count : k;
        const bool exact = p.E != nullptr && p.E[row] == 0.f;
        bool used64 = false;
        bool giant_tie = false;
        double dk64 = -1.0;  // FP64 distance placed at position kk - 1, when FP64 decided it
        if (!exact && kk > 0) {
            // near(i): positions i and i+1 cannot be ordered by their FP32 values
            auto near = [&](int i) -> bool {
                const float a = key_val(K[i]), b = key_val(K[i + 1]);
                return (b - a) <= TIE_REL * b;
            };
            bool any = false;
            for (int i = static_cast<int>(lane); i < kk && i + 1 < count; i += 32) any |= near(i);
            any = __any_sync(0xffffffffu, any);
            if (any) {
                used64 = true;
                int s = 0;
                while (s < kk) {
                    // group [s, e]: maximal run with near(s..e-1)
                    int e = s;
                    while (e + 1 < count && near(e)) ++e;
                    const int g = e - s + 1;
                    if (g > TIE_MAX) {
                        giant_tie = true;  // left unordered: the row is reported uncertified
                    } else if (g > 1) {
                        for (int m = s; m <= e; ++m) {
                            const uint32_t j = key_idx(K[m]);
                            const double v = sqdist_fp64(q, p.C + static_cast<int64_t>(j) * d, d);
                            if (lane == 0) T64[m - s] = v;
                        }
                        __syncwarp();
                        // rank every member by (FP64 distance, index) and place it; its key
                        // carries the FP64 distance rounded to FP32 (the output precision)
                        uint64_t my_key[TIE_MAX / 32];
                        int my_pos[TIE_MAX / 32];
                        int nm = 0;
                        for (int m = s + static_cast<int>(lane); m <= e; m += 32, ++nm) {
                            const double vm = T64[m - s];
                            const uint32_t jm = key_idx(K[m]);
                            int rank = 0;
                            for (int o = s; o <= e; ++o) {
                                const double vo = T64[o - s];
                                const uint32_t jo = key_idx(K[o]);
                                rank += (vo < vm || (vo == vm && jo < jm)) ? 1 : 0;
                            }
                            my_key[nm] = make_key(static_cast<float>(vm), jm);
                            my_pos[nm] = s + rank;
                            if (s + rank == kk - 1) dk64 = vm;
                        }
                        __syncwarp();
                        for (int t = 0; t < nm; ++t) K[my_pos[t]] = my_key[t];
                        __syncwarp();
                    }
                    s = e + 1;
                }
            }
        }

        // 3. outputs and certificate
        const int64_t ob = row * static_cast<int64_t>(k);
        for (int i = static_cast<int>(lane); i < k; i += 32) {
            if (i < kk) {
                p.out_idx[ob + i] = static_cast<int32_t>(key_idx(K[i]));
                p.out_dist[ob + i] = key_val(K[i]);
            } else {
                p.out_idx[ob + i] = -1;
                p.out_dist[ob + i] = F_INF;
            }
        }
        const bool truncated = (flags & ROW_TRUNCATED) || spec_cut;
        bool certified = kk == k && !(flags & ROW_SELECT_ERROR) && !giant_tie;
        if (certified && truncated && !exact) {
            // every left-out point has d' >= value(bound), so d2 >= value(bound) + |q|^2 - E
            double qn2 = 0.0;
            for (int t = static_cast<int>(lane); t < d; t += 32) qn2 = fma((double)q[t], (double)q[t], qn2);
            qn2 = warp_sum_d(qn2);
            // the lane that placed position kk - 1 in FP64 (if any) holds its distance
            const double dk64_w = __shfl_sync(0xffffffffu, dk64, __ffs(__ballot_sync(0xffffffffu, dk64 >= 0.0)) - 1);
            const bool have64 = __any_sync(0xffffffffu, dk64 >= 0.0);
            const double dk = have64 ? dk64_w : (double)key_val(K[kk - 1]) * (1.0 + 0x1p-19);
            const double bnd = (double)key_val(p.bound[row]);
            const double e = p.E ? (double)p.E[row] * (1.0 + 0x1p-10) : 0.0;
            const double slack = 0x1p-20 * (fabs(bnd) + qn2 + dk);
            certified = dk - qn2 < bnd - e - slack;
        }
        if (lane == 0) {
            p.row_status[row] = (certified ? 0u : ROW_UNCERTIFIED) | (used64 ? ROW_FP64 : 0u);
            atomicAdd(&blk_cnt[0], static_cast<unsigned long long>(count));
            if (used64) atomicAdd(&blk_cnt[1], 1ull);
            if (!certified) atomicAdd(&blk_cnt[2], 1ull);
            if (truncated) atomicAdd(&blk_cnt[3], 1ull);
            if (flags & ROW_THRESHOLD_MISS) atomicAdd(&blk_cnt[4], 1ull);
        }
    }
}

// Keys in a row's list (a raw list's count holds its two segments' lengths).
__device__ __forceinline__ int list_length(int raw, uint32_t flags) {
    return (flags & ROW_RAW_LIST) ? (raw & 0xffff) + (raw >> 16) : raw;
}

template <bool VEC>
__global__ void rerank_kernel(RerankParams p, int P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long blk_cnt[5];
    const int warp = static_cast<int>(threadIdx.x / 32);
    const int warps = static_cast<int>(blockDim.x / 32);
    const uint32_t lane = lane_id();
    if (threadIdx.x < 5) blk_cnt[threadIdx.x] = 0ull;
    __syncthreads();
    const int64_t row = static_cast<int64_t>(blockIdx.x) * warps + warp;
    if (row < p.M) {
        const int c = list_length(p.count[row], p.flags[row]);
        if (c >= p.count_min && c <= p.count_max) {
            uint64_t* K = reinterpret_cast<uint64_t*>(smem_raw) + static_cast<size_t>(warp) * (P + TIE_MAX);
            double* T64 = reinterpret_cast<double*>(K + P);
            rerank_row<VEC>(p, row, P, K, T64, blk_cnt, lane);
        }
    }
    flush_counters(p.counters, blk_cnt);
}

__device__ __forceinline__ int find_seg(const BatchSeg* segs, int32_t nseg, int64_t row) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].row0 <= row) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void rerank_batched_kernel(const BatchDev* __restrict__ probs, const BatchSeg* __restrict__ segs,
                                      int32_t nseg, int64_t rows, int P, int32_t count_min, int32_t count_max,
                                      RerankCounters* counters) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long blk_cnt[5];
    const int warp = static_cast<int>(threadIdx.x / 32);
    const int warps = static_cast<int>(blockDim.x / 32);
    const uint32_t lane = lane_id();
    if (threadIdx.x < 5) blk_cnt[threadIdx.x] = 0ull;
    __syncthreads();
    const int64_t row = static_cast<int64_t>(blockIdx.x) * warps + warp;
    if (row < rows) {
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
        const int64_t r = row - sg.row0;
        const int c = list_length(b.count[r], b.flags[r]);
        if (c >= count_min && c <= count_max) {
            uint64_t* K = reinterpret_cast<uint64_t*>(smem_raw) + static_cast<size_t>(warp) * (P + TIE_MAX);
            double* T64 = reinterpret_cast<double*>(K + P);
            const int Pp = pow2_ceil(b.cap > 32 ? b.cap : 32) < P ? pow2_ceil(b.cap > 32 ? b.cap : 32) : P;
            if (b.vec)
                rerank_row<true>(rp, r, Pp, K, T64, blk_cnt, lane);
            else
                rerank_row<false>(rp, r, Pp, K, T64, blk_cnt, lane);
        }
    }
    flush_counters(counters, blk_cnt);
}


}  // namespace

namespace {
cudaError_t launch_rerank_batched_range(const BatchDev* probs, const BatchSeg* segs, int32_t nseg, int64_t rows,
                                        int P, int32_t cmin, int32_t cmax, RerankCounters* counters,
                                        cudaStream_t st) {
    const size_t per_warp = static_cast<size_t>(P + TIE_MAX) * 8;
    int warps = static_cast<int>((64u * 1024u) / per_warp);
    if (warps > 8) warps = 8;
    if (warps < 1) warps = 1;
    const size_t smem = per_warp * warps;
    cudaError_t e = cudaFuncSetAttribute(rerank_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int64_t blocks = (rows + warps - 1) / warps;
    rerank_batched_kernel<<<static_cast<unsigned>(blocks), warps * 32, smem, st>>>(probs, segs, nseg, rows, P, cmin,
                                                                                   cmax, counters);
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
    for (int tier : {512, 1024}) {
        if (P <= tier) break;
        cudaError_t e = launch_rerank_batched_range(probs, segs, nseg, rows, tier, lo, tier, counters, st);
        if (e != cudaSuccess) return e;
        lo = tier + 1;
    }
    return launch_rerank_batched_range(probs, segs, nseg, rows, P, lo, INT32_MAX, counters, st);
}

namespace {
cudaError_t launch_rerank_range(RerankParams p, int P, int32_t cmin, int32_t cmax, cudaStream_t st) {
    p.count_min = cmin;
    p.count_max = cmax;
    const size_t per_warp = static_cast<size_t>(P + TIE_MAX) * 8;
    int warps = static_cast<int>((64u * 1024u) / per_warp);
    if (warps > 8) warps = 8;
    if (warps < 1) warps = 1;
    const size_t smem = per_warp * warps;
    const bool vec = (p.d % 4 == 0) && (reinterpret_cast<uintptr_t>(p.Q) % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(p.C) % 16 == 0);
    auto kern = vec ? rerank_kernel<true> : rerank_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int64_t blocks = (p.M + warps - 1) / warps;
    kern<<<static_cast<unsigned>(blocks), warps * 32, smem, st>>>(p, P);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_rerank(const RerankParams& p, cudaStream_t st) {
    if (p.M <= 0) return cudaSuccess;
    const int P = pow2_ceil(p.cap > 32 ? p.cap : 32);
    int lo = INT32_MIN;
    for (int tier : {512, 1024}) {
        if (P <= tier) break;
        cudaError_t e = launch_rerank_range(p, tier, lo, tier, st);
        if (e != cudaSuccess) return e;
        lo = tier + 1;
    }
    return launch_rerank_range(p, P, lo, INT32_MAX, st);
}

}  // namespace knn
