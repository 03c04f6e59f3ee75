// Last-resort exact rows in FP64: used only for rows that no faster path could
// certify (for example a row where more than a hundred points tie within FP32
// rounding at the k-th distance). One block per row: the FP64 value of every corpus
// point (the direct-difference squared distance, or the cosine / Pearson similarity)
// as an order-preserving 64-bit key (smaller key = nearer), an 8-pass radix select on
// the keys for the k-th smallest, then the points below it plus the lowest-index points
// equal to it, sorted by (key, index).
#include "common.cuh"
#include "internal.h"

namespace knn {
namespace {

constexpr int XT = 256;
constexpr int XMAXK = 2048;

// Order-preserving map of a double to uint64: a < b <=> key(a) < key(b); -0 is folded onto
// +0 so that equal values have equal keys.
__device__ __forceinline__ unsigned long long key_of(double v) {
    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v == 0.0 ? 0.0 : v));
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double value_of(unsigned long long k) {
    const unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double(static_cast<long long>(u));
}

struct SimStats {
    int32_t centered;
    const double* qmean;
    const double* qnorm;
    const double* cmean;
    const double* cnorm;
};

// METRIC 0: squared Euclidean distance, ascending; 1: similarity, descending (key of -s).
template <int METRIC>
__global__ void __launch_bounds__(XT) exact_rows_kernel(const float* __restrict__ Q, const float* __restrict__ C,
                                                        int64_t N, int32_t d, int32_t k, int32_t exclude_self,
                                                        SimStats ss, const int32_t* __restrict__ rows,
                                                        double* __restrict__ scratch, int32_t* __restrict__ out_idx,
                                                        float* __restrict__ out_dist) {
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long prefix_sh;
    __shared__ int rank_sh;
    __shared__ int n_lt_sh;
    __shared__ unsigned long long sel_key[XMAXK];  // keys, sorted later with the index
    __shared__ int sel_idx[XMAXK];
    __shared__ int n_sel;

    const int64_t row = rows[blockIdx.x];
    const float* q = Q + row * d;
    unsigned long long* dist = reinterpret_cast<unsigned long long*>(scratch + static_cast<int64_t>(blockIdx.x) * N);
    const int warp = static_cast<int>(threadIdx.x / 32), lane = static_cast<int>(threadIdx.x % 32);
    const double mq = (METRIC == 1 && ss.centered) ? ss.qmean[row] : 0.0;

    for (int64_t j = warp; j < N; j += XT / 32) {
        double s = 0.0;
        const float* c = C + j * d;
        if (METRIC == 0) {
            for (int t = lane; t < d; t += 32) {
                const double diff = static_cast<double>(q[t]) - static_cast<double>(c[t]);
                s = fma(diff, diff, s);
            }
        } else {
            const double mc = ss.centered ? ss.cmean[j] : 0.0;
            for (int t = lane; t < d; t += 32)
                s = fma(static_cast<double>(q[t]) - mq, static_cast<double>(c[t]) - mc, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            unsigned long long key;
            if (exclude_self && j == row) {
                key = ~0ull;
            } else if (METRIC == 0) {
                key = key_of(s);
            } else {
                key = key_of(-(s / (ss.qnorm[row] * ss.cnorm[j])));
            }
            dist[j] = key;
        }
    }
    __syncthreads();

    // radix select of the k-th smallest bit pattern
    if (threadIdx.x == 0) {
        prefix_sh = 0ull;
        rank_sh = k - 1;
    }
    __syncthreads();
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        const unsigned long long hi_mask = pass == 0 ? 0ull : (~0ull << (shift + 8));
        for (int b = threadIdx.x; b < 256; b += XT) hist[b] = 0u;
        __syncthreads();
        const unsigned long long prefix = prefix_sh;
        for (int64_t j = threadIdx.x; j < N; j += XT) {
            const unsigned long long u = dist[j];
            if ((u & hi_mask) == prefix) atomicAdd(&hist[(u >> shift) & 0xffu], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int r = rank_sh;
            int b = 0;
            while (b < 255 && r >= static_cast<int>(hist[b])) {
                r -= static_cast<int>(hist[b]);
                ++b;
            }
            rank_sh = r;
            prefix_sh = prefix | (static_cast<unsigned long long>(b) << shift);
        }
        __syncthreads();
    }
    const unsigned long long vk = prefix_sh;
    // points strictly below the k-th value (fewer than k of them), any order
    if (threadIdx.x == 0) n_sel = 0;
    __syncthreads();
    for (int64_t j = threadIdx.x; j < N; j += XT) {
        const unsigned long long u = dist[j];
        if (u < vk) {
            const int s = atomicAdd(&n_sel, 1);
            if (s < XMAXK) {
                sel_key[s] = u;
                sel_idx[s] = static_cast<int>(j);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) n_lt_sh = n_sel;
    __syncthreads();
    // then the lowest-index points equal to it, in index order (one warp, ballots)
    if (warp == 0) {
        int have = n_lt_sh;
        for (int64_t base = 0; base < N && have < k; base += 32) {
            const int64_t j = base + lane;
            const bool eq = j < N && dist[j] == vk;
            const unsigned int b = __ballot_sync(0xffffffffu, eq);
            const int pos = have + __popc(b & ((1u << lane) - 1u));
            if (eq && pos < k && pos < XMAXK) {
                sel_key[pos] = vk;
                sel_idx[pos] = static_cast<int>(j);
            }
            have += __popc(b);
        }
    }
    __syncthreads();
    // sort the k selected by (distance, index): rank counting (k <= XMAXK)
    const int kk = k < XMAXK ? k : XMAXK;
    for (int i = threadIdx.x; i < kk; i += XT) {
        const unsigned long long ui = sel_key[i];
        const int ji = sel_idx[i];
        int r = 0;
        for (int o = 0; o < kk; ++o) {
            const unsigned long long uo = sel_key[o];
            r += (uo < ui || (uo == ui && sel_idx[o] < ji)) ? 1 : 0;
        }
        out_idx[row * k + r] = ji;
        const double v = value_of(ui);
        out_dist[row * k + r] = static_cast<float>(METRIC == 0 ? v : -v);
    }
}

}  // namespace

cudaError_t launch_exact_rows_fp64(const float* Q, const float* C, int64_t N, int32_t d, int32_t k,
                                   int32_t exclude_self, const int32_t* rows, int32_t nrows, double* scratch,
                                   int32_t* out_idx, float* out_dist, cudaStream_t st) {
    if (nrows <= 0) return cudaSuccess;
    if (k > XMAXK) return cudaErrorInvalidValue;
    exact_rows_kernel<0><<<nrows, XT, 0, st>>>(Q, C, N, d, k, exclude_self, SimStats{}, rows, scratch, out_idx,
                                               out_dist);
    return cudaGetLastError();
}

cudaError_t launch_exact_rows_sim_fp64(const float* Q, const float* C, int64_t N, int32_t d, int32_t k,
                                       int32_t exclude_self, int32_t centered, const double* qmean,
                                       const double* qnorm, const double* cmean, const double* cnorm,
                                       const int32_t* rows, int32_t nrows, double* scratch, int32_t* out_idx,
                                       float* out_val, cudaStream_t st) {
    if (nrows <= 0) return cudaSuccess;
    if (k > XMAXK) return cudaErrorInvalidValue;
    const SimStats ss{centered, qmean, qnorm, cmean, cnorm};
    exact_rows_kernel<1><<<nrows, XT, 0, st>>>(Q, C, N, d, k, exclude_self, ss, rows, scratch, out_idx, out_val);
    return cudaGetLastError();
}

}  // namespace knn
