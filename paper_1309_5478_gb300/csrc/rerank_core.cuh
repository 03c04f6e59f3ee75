// Exact re-rank of one row's candidate list by one warp (device code, header-only so
// that the re-rank kernels and the fused kernel's re-rank warps share it).
//
// The candidate lists come from the selection (fused or not) on approximate
// ranking values d'_ij = |c_j|^2 - 2 q_i.c_j (Methods, "Distance calculation").
// Here every candidate's squared distance is recomputed in the direct difference
// form sum_t (q_t - c_t)^2, which has no cancellation:
//   - 8, 16 or 32 lanes share a candidate (by dimension); each lane adds the eight
//     products of two 16-byte pieces with FMAs and folds that sum into a (sum, error)
//     pair with Knuth's TwoSum, then rounds its pair to one float, and the lanes' floats
//     are summed by a shuffle tree. Every term is non-negative, so each rounding adds at
//     most one unit of the total: the relative error is at most 2 units in the last place
//     for the rounded differences, 8 for the sums of eight products, 1 for a lane's pair
//     and 5 for the tree over 32 lanes (3 over 8), 16 in all: at most 2^-20.
//   - candidates are taken in ascending approximate order. Once the first k are exact,
//     the largest of them bounds the exact k-th distance of the row from above; a
//     candidate whose approximate value is more than E_i above that bound (with
//     slack for the FP32 roundings) cannot be among the k nearest, and neither can any
//     later one, so the rest of the list is not gathered.
//   - the list is sorted by (FP32 distance, index). Neighbours in the sorted list that
//     are within 2^-19 (relative) of each other around the first k positions form
//     near-tie groups; their distances are recomputed in FP64 and the group re-sorted
//     by (FP64 distance, index). FP64 therefore decides only the order of points whose
//     FP32 distances cannot be told apart.
//   - a row whose list was truncated is certified only if the k-th exact distance is
//     below the smallest value any left-out point can have, bound - E (in d' scale).
//   - for every candidate it evaluates, the re-rank measures |approximate - exact| of d'
//     against the row's bound E_i; the largest ratio is reported, so the bound that every
//     certificate rests on is checked on the data at hand.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "select_core.cuh"

namespace knn {

constexpr float TIE_REL = 0x1p-19f;
// Members of one near-tie group settled in FP64 at most (a larger group is left unordered
// and its row reported uncertified).
constexpr int TIE_MAX = 128;
// Odd-even passes tried on a list in approximate order before it is sorted in full.
constexpr int SETTLE_PASSES = 32;

// Per-warp (or per-block) counters of the re-rank, in shared memory; flushed into
// RerankCounters by flush_rerank_counts.
enum RerankCount : int {
    RC_CANDIDATES = 0,
    RC_FP64_ROWS,
    RC_UNCERTIFIED,
    RC_TRUNCATED,
    RC_THRESHOLD_MISS,
    RC_ERR_RATIO,  // float bits of the largest |approximate - exact| / E (non-negative: unsigned max)
    RC_ROWS,       // rows re-ranked
    RC_COUNT
};

// The squares of two 16-byte pieces (eight differences, one rounding each) summed by a
// multiply and seven FMAs, then added to the lane's (sum, error) pair by TwoSum.
__device__ __forceinline__ void group_sum8(float4 q0, float4 c0, float4 q1, float4 c1, float& s, float& e) {
    const float d0 = q0.x - c0.x, d1 = q0.y - c0.y, d2 = q0.z - c0.z, d3 = q0.w - c0.w;
    const float d4 = q1.x - c1.x, d5 = q1.y - c1.y, d6 = q1.z - c1.z, d7 = q1.w - c1.w;
    float g = d0 * d0;
    g = fmaf(d1, d1, g);
    g = fmaf(d2, d2, g);
    g = fmaf(d3, d3, g);
    g = fmaf(d4, d4, g);
    g = fmaf(d5, d5, g);
    g = fmaf(d6, d6, g);
    g = fmaf(d7, d7, g);
    float t, err;
    two_sum(s, g, t, err);
    s = t;
    e += err;
}

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

__device__ __forceinline__ float4 load4(const float* __restrict__ p, int t, int d, bool vec) {
    if (vec) return __ldg(reinterpret_cast<const float4*>(p + t));
    float4 a;
    a.x = p[t];
    a.y = t + 1 < d ? p[t + 1] : 0.f;
    a.z = t + 2 < d ? p[t + 2] : 0.f;
    a.w = t + 3 < d ? p[t + 3] : 0.f;
    return a;
}

// Sum over an aligned group of G lanes of each lane's (sum, error) pair rounded to one
// float (plain tree: the partial sums are non-negative, one rounding per level); every
// lane of the group returns the group's total.
template <int G>
__device__ __forceinline__ float group_fold_sum(float s, float e) {
    float v = s + e;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Squared distances of the query q to NC candidate rows at once (NC rows of loads in flight
// per lane); every lane returns the results. VEC: d % 4 == 0 and 16-byte aligned rows.
template <bool VEC, int NC>
__device__ __forceinline__ void sqdist_multi(const float* __restrict__ q, const float* const (&c)[NC], int d,
                                             float (&r)[NC]) {
    const uint32_t lane = lane_id();
    float s[NC], e[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) s[i] = e[i] = 0.f;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
    for (int t = static_cast<int>(lane) * 4; t < d; t += 256) {
        const bool two = t + 128 < d;
        const float4 a0 = load4(q, t, d, VEC);
        const float4 a1 = two ? load4(q, t + 128, d, VEC) : z;
        float4 b0[NC], b1[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            b0[i] = load4(c[i], t, d, VEC);
            b1[i] = two ? load4(c[i], t + 128, d, VEC) : z;
        }
#pragma unroll
        for (int i = 0; i < NC; ++i) group_sum8(a0, b0[i], a1, b1[i], s[i], e[i]);
    }
#pragma unroll
    for (int i = 0; i < NC; ++i) r[i] = group_fold_sum<32>(s[i], e[i]);
}

// |q|^2 with the same compensated summation (relative error below 2^-20).
template <bool VEC>
__device__ __forceinline__ float sqnorm_comp(const float* __restrict__ q, int d) {
    const uint32_t lane = lane_id();
    float s = 0.f, e = 0.f;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int t = static_cast<int>(lane) * 4; t < d; t += 128) group_sum(load4(q, t, d, VEC), z, s, e);
    return warp_reduce_pair(s, e);
}

__device__ __forceinline__ double sqdist_fp64(const float* __restrict__ q, const float* __restrict__ c, int d) {
    double s = 0.0;
    for (int t = static_cast<int>(lane_id()); t < d; t += 32) {
        const double diff = static_cast<double>(q[t]) - static_cast<double>(c[t]);
        s = fma(diff, diff, s);
    }
    return warp_sum_d(s);
}

// Keys in a row's list (a raw list's count holds its two segments' lengths).
__device__ __forceinline__ int list_length(int raw, uint32_t flags) {
    return (flags & ROW_RAW_LIST) ? (raw & 0xffff) + (raw >> 16) : raw;
}

// Keys of a row's inbox (symmetric graph form) that the re-rank reads: at most cap_in.
__device__ __forceinline__ int inbox_length(const RerankParams& p, int64_t row) {
    if (!p.inbox_cnt) return 0;
    const int c = p.inbox_cnt[row];
    return c < p.cap_in ? c : p.cap_in;
}

// Keys the re-rank of a row sorts: its list and its inbox.
__device__ __forceinline__ int row_keys(const RerankParams& p, int64_t row) {
    return list_length(p.count[row], p.flags[row]) + inbox_length(p, row);
}

// Exact keys for positions [lo, hi) of K (approximate keys in, exact keys out), NC
// candidates at a time, each shared by the whole warp; err_max collects
// |approximate + qn2 - exact| / E (E > 0).
template <bool VEC, int NC>
__device__ __forceinline__ void exact_keys_warp(const RerankParams& p, const float* __restrict__ q, uint64_t* K, int lo,
                                           int hi, float qn2, float inv_e, float& err_max, uint32_t lane) {
    const int d = p.d;
    int c = lo;
    for (; c + NC <= hi; c += NC) {
        uint32_t j[NC];
        float a[NC];
        const float* cp[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            const uint64_t key = K[c + i];
            j[i] = key_idx(key);
            a[i] = key_val(key);
            cp[i] = p.C + static_cast<int64_t>(j[i]) * d;
        }
        float r[NC];
        sqdist_multi<VEC, NC>(q, cp, d, r);
#pragma unroll
        for (int i = 0; i < NC; ++i) err_max = fmaxf(err_max, fabsf((a[i] + qn2) - r[i]) * inv_e);
        // every lane has read these keys before the reduction's shuffles: lane 0 may overwrite them
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < NC; ++i) K[c + i] = make_key(r[i], j[i]);
        }
    }
    for (; c < hi; ++c) {
        const uint64_t key = K[c];
        const float* cp[1] = {p.C + static_cast<int64_t>(key_idx(key)) * d};
        float r[1];
        sqdist_multi<VEC, 1>(q, cp, d, r);
        err_max = fmaxf(err_max, fabsf((key_val(key) + qn2) - r[0]) * inv_e);
        if (lane == 0) K[c] = make_key(r[0], key_idx(key));
    }
    __syncwarp();
}

// Exact keys for positions [lo, hi) of K (approximate keys in, exact keys out), with
// the warp split into 32 / G groups of G lanes; err_max collects
// |approximate + qn2 - exact| / E (E > 0) and is warp-uniform on return. A group takes NC
// candidates at a time, each lane reading one 16-byte piece of each candidate row per
// step, so one pass evaluates 32 / G * NC candidates and a distance's reduction takes
// log2(G) shuffle levels.
template <bool VEC, int G, int NC>
__device__ __forceinline__ void exact_keys_g(const RerankParams& p, const float* __restrict__ q, uint64_t* K, int lo,
                                             int hi, float qn2, float inv_e, float& err_max, uint32_t lane) {
    constexpr int PER = (32 / G) * NC;
    const int d = p.d;
    const int g = static_cast<int>(lane) / G;
    const int gl = static_cast<int>(lane) % G;
    for (int c = lo; c < hi; c += PER) {
        uint32_t j[NC];
        float a[NC];
        const float* cp[NC];
        bool live[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            const int pos = c + g * NC + i;
            live[i] = pos < hi;
            const uint64_t key = K[live[i] ? pos : lo];
            j[i] = key_idx(key);
            a[i] = key_val(key);
            cp[i] = p.C + static_cast<int64_t>(j[i]) * d;
        }
        float s[NC], e[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) s[i] = e[i] = 0.f;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
        for (int t = gl * 4; t < d; t += 8 * G) {
            const bool two = t + 4 * G < d;
            const float4 qa = load4(q, t, d, VEC);
            const float4 qb = two ? load4(q, t + 4 * G, d, VEC) : z;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                float4 b0 = z, b1 = z;
                if (live[i]) {
                    b0 = load4(cp[i], t, d, VEC);
                    if (two) b1 = load4(cp[i], t + 4 * G, d, VEC);
                }
                group_sum8(qa, b0, qb, b1, s[i], e[i]);
            }
        }
        float r[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) r[i] = group_fold_sum<G>(s[i], e[i]);
#pragma unroll
        for (int i = 0; i < NC; ++i)
            if (live[i]) err_max = fmaxf(err_max, fabsf((a[i] + qn2) - r[i]) * inv_e);
        // every lane has read these keys before the reduction's shuffles: the group's first
        // lane may overwrite its group's keys
        if (gl == 0) {
#pragma unroll
            for (int i = 0; i < NC; ++i)
                if (live[i]) K[c + g * NC + i] = make_key(r[i], j[i]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) err_max = fmaxf(err_max, __shfl_xor_sync(0xffffffffu, err_max, o));
    __syncwarp();
}

// Lanes per candidate by dimension: short rows are shared by fewer lanes (more candidates
// at once, fewer shuffle levels); above d = 256 the whole warp reads each row in 512-byte
// steps (exact_keys_warp), which keeps the gathers in long bursts per row (measured on
// GB300: with groups of 8 lanes the 262144 x 1024 graph's re-rank took 33 ms instead of
// 19.6 ms, while the d = 64 problems of a batch went from 15.8 to 13.1 ms).
__host__ __device__ constexpr int rerank_group(int d) { return d <= 128 ? 8 : (d <= 256 ? 16 : 32); }

// G: lanes per candidate (32: exact_keys_warp), or 0 to choose by p.d at run time among
// the grouped forms (kernels whose rows have several dimensions; fewer registers than with
// exact_keys_warp among them). exact_keys_g<32> and exact_keys_warp do the same operations
// on every candidate, so every kernel gives a row bit-identical distances.
template <bool VEC, int G, int NC>
__device__ __forceinline__ void exact_keys(const RerankParams& p, const float* __restrict__ q, uint64_t* K, int lo,
                                           int hi, float qn2, float inv_e, float& err_max, uint32_t lane) {
    if constexpr (G == 32) {
        exact_keys_warp<VEC, NC>(p, q, K, lo, hi, qn2, inv_e, err_max, lane);
    } else if constexpr (G != 0) {
        exact_keys_g<VEC, G, NC>(p, q, K, lo, hi, qn2, inv_e, err_max, lane);
    } else {
        if (p.d <= 128)
            exact_keys_g<VEC, 8, NC>(p, q, K, lo, hi, qn2, inv_e, err_max, lane);
        else if (p.d <= 256)
            exact_keys_g<VEC, 16, NC>(p, q, K, lo, hi, qn2, inv_e, err_max, lane);
        else
            exact_keys_g<VEC, 32, NC>(p, q, K, lo, hi, qn2, inv_e, err_max, lane);
    }
}

// One warp re-ranks row `row` of p; K is the warp's shared-memory array of P keys
// (P >= the row's list length, a power of two) and T64 its TIE_MAX doubles for one
// near-tie group; cnt the warp's RC_COUNT counters (shared memory).
template <bool VEC, int NC, int G = 0>
__device__ __forceinline__ void rerank_row(const RerankParams& p, int64_t row, int P, uint64_t* K, double* T64,
                                           unsigned long long* cnt, uint32_t lane) {
    const int raw = p.count[row];
    const uint32_t flags = p.flags[row];
    const float* q = p.Q + row * static_cast<int64_t>(p.d);
    const uint64_t* cand = p.cand + row * static_cast<int64_t>(p.cap);
    const int d = p.d;
    const float erow = p.E ? p.E[row] : 0.f;

    // 0. the row's candidate keys into K. A raw list (every key <= bound, in a front and
    //    a back segment) is first reduced to the band of its approximate values, as the
    //    select does: sorted, then the keys <= min(bound, max(key_(k+m), ceiling(v_(k) +
    //    2E))) kept. A row whose bound came from a speculative threshold is truncated
    //    there when that band reaches beyond it.
    //    In the symmetric graph form the row's inbox (keys of the transposed pairs, every one
    //    at or below the row's bound is there unless the inbox overflowed) joins the list.
    int count;
    bool spec_cut = false;
    bool sorted = false;
    bool lost = false;  // the inbox overflowed: keys below the bound may be missing
    if (flags & ROW_RAW_LIST) {
        const int n0 = raw & 0xffff, nl = n0 + (raw >> 16);
        const int nin = inbox_length(p, row);
        lost = p.inbox_cnt != nullptr && p.inbox_cnt[row] > p.cap_in;
        const uint64_t* inbox = p.inbox ? p.inbox + row * static_cast<int64_t>(p.cap_in) : nullptr;
        const int n = nl + nin;
        const int Pn = pow2_ceil(n > 32 ? n : 32) < P ? pow2_ceil(n > 32 ? n : 32) : P;
        for (int i = static_cast<int>(lane); i < Pn; i += 32)
            K[i] = i < n0 ? cand[i] : (i < nl ? cand[p.cap - 1 - (i - n0)] : (i < n ? inbox[i - nl] : KEY_MAX));
        __syncwarp();
        warp_bitonic_sort_smem(K, Pn);
        const int kk = n < p.k ? n : p.k;
        uint64_t band = KEY_MAX;
        if (n >= p.km && n > 0) {
            band = K[p.km - 1];
            const float window = 2.f * erow;
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
        sorted = true;
    } else {
        count = raw;
        for (int i = static_cast<int>(lane); i < count; i += 32) K[i] = cand[i];
    }
    __syncwarp();

    const int k = p.k;
    const int kk = count < k ? count : k;
    // the early stop needs the list in ascending approximate order and a bound
    const bool can_stop = p.E != nullptr && kk == k && count > kk;
    if (can_stop && !sorted) {
        const int Pn = pow2_ceil(count > 32 ? count : 32) < P ? pow2_ceil(count > 32 ? count : 32) : P;
        for (int i = count + static_cast<int>(lane); i < Pn; i += 32) K[i] = KEY_MAX;
        __syncwarp();
        warp_bitonic_sort_smem(K, Pn);
    }
    const bool measure = erow > 0.f;
    const float qn2 = (can_stop || measure) ? sqnorm_comp<VEC>(q, d) : 0.f;
    const float inv_e = measure ? 1.f / erow : 0.f;
    float err_max = 0.f;

    // 1. direct-difference FP32 distances: the first k candidates, then the rest up to
    //    the first one that provably lies beyond the k-th exact distance
    exact_keys<VEC, G, NC>(p, q, K, 0, kk, qn2, inv_e, err_max, lane);
    int stop = count;
    if (can_stop) {
        float mx = 0.f;
        for (int i = static_cast<int>(lane); i < kk; i += 32) mx = fmaxf(mx, key_val(K[i]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        // exact k-th <= mx (1 + 2^-19); a candidate's exact d2 >= |q|^2 + approx - E, with
        // |q|^2 >= qn2 (1 - 2^-19): skip when that lower bound exceeds the upper one
        const double lim = static_cast<double>(mx) * (1.0 + 0x1p-18) - static_cast<double>(qn2) * (1.0 - 0x1p-18) +
                           static_cast<double>(erow) + 0x1p-40;
        int first = count;
        for (int i = kk + static_cast<int>(lane); i < count; i += 32)
            if (static_cast<double>(key_val(K[i])) > lim) {
                first = i;
                break;
            }
        stop = static_cast<int>(__reduce_min_sync(0xffffffffu, static_cast<uint32_t>(first)));
    }
    exact_keys<VEC, G, NC>(p, q, K, kk, stop, qn2, inv_e, err_max, lane);
    count = stop;

    // sort by exact distance. A list taken in ascending approximate order is off by the
    // approximation error only, a few positions: odd-even passes settle it. Otherwise (or
    // when the passes do not settle it) sort only the power of two that holds the list.
    const bool presorted = sorted || can_stop;
    if (!presorted || !warp_oddeven_settle(K, count, SETTLE_PASSES)) {
        const int Pc = pow2_ceil(count > 32 ? count : 32) < P ? pow2_ceil(count > 32 ? count : 32) : P;
        for (int i = count + static_cast<int>(lane); i < Pc; i += 32) K[i] = KEY_MAX;
        __syncwarp();
        warp_bitonic_sort_smem(K, Pc);
    }

    // 2. near ties around the first k positions, settled in FP64 (skipped when the
    //    inputs make FP32 exact: then equal values are true ties, already ordered by index)
    const bool exact = p.E != nullptr && erow == 0.f;
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
            // groups: maximal runs [s, e] with near(s..e-1), s < kk, found 32 positions a
            // ballot. Positions from `next` on still hold their sorted FP32 keys (a placed
            // group only rewrites its own positions), and next itself starts a run when
            // near(next) holds, the run before it having ended at next - 1.
            int next = 0;
            while (next < kk) {
                const int i = next + static_cast<int>(lane);
                const bool st = i < kk && i + 1 < count && near(i) && (i == next || !near(i - 1));
                const uint32_t sm = __ballot_sync(0xffffffffu, st);
                if (sm == 0u) {
                    next += 32;
                    continue;
                }
                const int s = next + __ffs(sm) - 1;
                int e = s;
                for (int b = s;; b += 32) {
                    const int j = b + static_cast<int>(lane);
                    const uint32_t em = __ballot_sync(0xffffffffu, !(j + 1 < count && near(j)));
                    if (em != 0u) {
                        e = b + __ffs(em) - 1;
                        break;
                    }
                }
                next = e + 1;
                const int g = e - s + 1;
                if (g > TIE_MAX) {
                    giant_tie = true;  // left unordered: the row is reported uncertified
                } else {
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
    // a list complete up to a bounding threshold answers exactly among the points within it,
    // with fewer than k of them when the bound holds fewer
    const bool bounded = (flags & ROW_BOUNDED) != 0u;
    bool certified = (kk == k || bounded) && !(flags & ROW_SELECT_ERROR) && !giant_tie && !lost;
    if (certified && truncated && !exact && !bounded) {
        // every left-out point has d' >= value(bound), so d2 >= value(bound) + |q|^2 - E
        double qn2d = 0.0;
        for (int t = static_cast<int>(lane); t < d; t += 32) qn2d = fma((double)q[t], (double)q[t], qn2d);
        qn2d = warp_sum_d(qn2d);
        // the lane that placed position kk - 1 in FP64 (if any) holds its distance
        const double dk64_w = __shfl_sync(0xffffffffu, dk64, __ffs(__ballot_sync(0xffffffffu, dk64 >= 0.0)) - 1);
        const bool have64 = __any_sync(0xffffffffu, dk64 >= 0.0);
        const double dk = have64 ? dk64_w : (double)key_val(K[kk - 1]) * (1.0 + 0x1p-19);
        const double bnd = (double)key_val(p.bound[row]);
        const double e = p.E ? (double)erow * (1.0 + 0x1p-10) : 0.0;
        const double slack = 0x1p-20 * (fabs(bnd) + qn2d + dk);
        certified = dk - qn2d < bnd - e - slack;
    }
    if (lane == 0) {
        p.row_status[row] = (certified ? 0u : ROW_UNCERTIFIED) | (used64 ? ROW_FP64 : 0u) | ROW_RERANKED;
        if (!certified && p.uncertified) atomicAdd(p.uncertified, 1u);
        cnt[RC_CANDIDATES] += static_cast<unsigned long long>(count);
        if (used64) cnt[RC_FP64_ROWS] += 1ull;
        if (!certified) cnt[RC_UNCERTIFIED] += 1ull;
        if (truncated) cnt[RC_TRUNCATED] += 1ull;
        if (flags & ROW_THRESHOLD_MISS) cnt[RC_THRESHOLD_MISS] += 1ull;
        const unsigned long long eb = __float_as_uint(err_max);
        if (eb > cnt[RC_ERR_RATIO]) cnt[RC_ERR_RATIO] = eb;
        cnt[RC_ROWS] += 1ull;
    }
}

// Adds per-warp counters (one lane) to the call's counters in global memory.
__device__ __forceinline__ void flush_rerank_counts(RerankCounters* counters, const unsigned long long* cnt,
                                                    bool in_sweep) {
    if (!counters) return;
    if (cnt[RC_CANDIDATES]) atomicAdd(&counters->candidates, cnt[RC_CANDIDATES]);
    if (cnt[RC_FP64_ROWS]) atomicAdd(&counters->fp64_rows, cnt[RC_FP64_ROWS]);
    if (cnt[RC_UNCERTIFIED]) atomicAdd(&counters->uncertified, cnt[RC_UNCERTIFIED]);
    if (cnt[RC_TRUNCATED]) atomicAdd(&counters->truncated, cnt[RC_TRUNCATED]);
    if (cnt[RC_THRESHOLD_MISS]) atomicAdd(&counters->threshold_miss, cnt[RC_THRESHOLD_MISS]);
    if (cnt[RC_ERR_RATIO]) atomicMax(&counters->max_err_ratio, cnt[RC_ERR_RATIO]);
    if (in_sweep && cnt[RC_ROWS]) atomicAdd(&counters->rows_in_sweep, cnt[RC_ROWS]);
}

}  // namespace knn
