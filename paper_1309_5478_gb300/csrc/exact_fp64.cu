// Last-resort exact rows in FP64: used only for rows that no faster path could
// certify (for example a row where more than a hundred points tie within FP32
// rounding at the k-th distance). One block per row: FP64 direct-difference
// distances to every corpus point, an 8-pass radix select on the FP64 bit pattern
// (non-negative doubles order like their bits) for the k-th smallest value, then the
// points below it plus the lowest-index points equal to it, sorted by (distance, index).
#include "common.cuh"
#include "internal.h"

namespace knn {
namespace {

constexpr int XT = 256;
constexpr int XMAXK = 2048;

__global__ void __launch_bounds__(XT) exact_rows_kernel(const float* __restrict__ Q, const float* __restrict__ C,
                                                        int64_t N, int32_t d, int32_t k, int32_t exclude_self,
                                                        const int32_t* __restrict__ rows, double* __restrict__ scratch,
                                                        int32_t* __restrict__ out_idx, float* __restrict__ out_dist) {
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long prefix_sh;
    __shared__ int rank_sh;
    __shared__ int n_lt_sh;
    __shared__ unsigned long long sel_key[XMAXK];  // (bits of double) sorted later with the index
    __shared__ int sel_idx[XMAXK];
    __shared__ int n_sel;

    const int64_t row = rows[blockIdx.x];
    const float* q = Q + row * d;
    double* dist = scratch + static_cast<int64_t>(blockIdx.x) * N;
    const int warp = static_cast<int>(threadIdx.x / 32), lane = static_cast<int>(threadIdx.x % 32);

    for (int64_t j = warp; j < N; j += XT / 32) {
        double s = 0.0;
        const float* c = C + j * d;
        for (int t = lane; t < d; t += 32) {
            const double diff = static_cast<double>(q[t]) - static_cast<double>(c[t]);
            s = fma(diff, diff, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) dist[j] = (exclude_self && j == row) ? __longlong_as_double(0x7ff0000000000000ll) : s;
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
            const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(dist[j]));
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
        const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(dist[j]));
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
            const bool eq = j < N && static_cast<unsigned long long>(__double_as_longlong(dist[j])) == vk;
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
        out_dist[row * k + r] = static_cast<float>(__longlong_as_double(static_cast<long long>(ui)));
    }
}

}  // namespace

cudaError_t launch_exact_rows_fp64(const float* Q, const float* C, int64_t N, int32_t d, int32_t k,
                                   int32_t exclude_self, const int32_t* rows, int32_t nrows, double* scratch,
                                   int32_t* out_idx, float* out_dist, cudaStream_t st) {
    if (nrows <= 0) return cudaSuccess;
    if (k > XMAXK) return cudaErrorInvalidValue;
    exact_rows_kernel<<<nrows, XT, 0, st>>>(Q, C, N, d, k, exclude_self, rows, scratch, out_idx, out_dist);
    return cudaGetLastError();
}

}  // namespace knn
