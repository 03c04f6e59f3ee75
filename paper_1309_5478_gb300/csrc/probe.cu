// Band probe: how many candidates per row the band rule of the tensor-core form keeps.
//
// The fused selection keeps, for every row, the keys below T = max(v_(k+m), v_(k) + 2E)
// (E the row's bound on the reduced-precision error of d'). When the inputs make that
// band wide (d' values crowded within 2E of the k-th), a list capacity sized for k + m
// overflows again and again and ends truncated. This kernel counts the band of a few
// sampled rows from their FP32 d' values, so the host can size the list before the
// fused launch. It also reports each sampled row's band edge as a squared distance,
// T + |q|^2, from which the host derives a speculative start threshold.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace knn {
namespace {

__global__ void band_count_kernel(const float* __restrict__ D, int64_t N, int64_t ldd, const float* __restrict__ vals,
                                  int32_t k, int32_t km, const float* __restrict__ E,
                                  const int32_t* __restrict__ self_col, const float* __restrict__ qnorm2,
                                  const int32_t* __restrict__ rows, int32_t* __restrict__ out_count,
                                  int32_t* __restrict__ out_count4, float* __restrict__ out_edge) {
    const int64_t i = blockIdx.x;
    const float* v = vals + i * km;
    const float T = fmaxf(v[km - 1], v[k - 1] + 2.f * E[i]);
    // a list built on approximate values (each within E) keeps keys up to exact v_k + 4E
    const float T4 = fmaxf(v[km - 1], v[k - 1] + 4.f * E[i]);
    const float* row = D + i * ldd;
    const int64_t self = self_col ? self_col[i] : -1;
    int c = 0, c4 = 0;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
        c += (row[j] <= T && j != self) ? 1 : 0;
        c4 += (row[j] <= T4 && j != self) ? 1 : 0;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    c4 = __reduce_add_sync(0xffffffffu, c4);
    __shared__ int part[32], part4[32];
    if ((threadIdx.x & 31u) == 0) {
        part[threadIdx.x / 32] = c;
        part4[threadIdx.x / 32] = c4;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0, s4 = 0;
        for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) {
            s += part[w];
            s4 += part4[w];
        }
        out_count[i] = s;
        if (out_count4) out_count4[i] = s4;
        if (out_edge) out_edge[i] = T + qnorm2[rows[i]];
    }
}

// Keys of each sampled row at or below a squared distance t (other than the row itself): the
// transposed pairs the symmetric form would send to that row's inbox, at most.
__global__ void count_le_kernel(const float* __restrict__ D, int64_t N, int64_t ldd, float t,
                                const float* __restrict__ qnorm2, const int32_t* __restrict__ rows,
                                const int32_t* __restrict__ self_col, int32_t* __restrict__ out) {
    const int64_t i = blockIdx.x;
    const float lim = t - qnorm2[rows[i]];
    const float* row = D + i * ldd;
    const int64_t self = self_col ? self_col[i] : -1;
    int c = 0;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) c += (row[j] <= lim && j != self) ? 1 : 0;
    c = __reduce_add_sync(0xffffffffu, c);
    __shared__ int part[32];
    if ((threadIdx.x & 31u) == 0) part[threadIdx.x / 32] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) s += part[w];
        out[i] = s;
    }
}

}  // namespace

cudaError_t launch_count_le(const float* D, int64_t rows, int64_t N, int64_t ldd, float t, const float* qnorm2,
                            const int32_t* row_ids, const int32_t* self_col, int32_t* out, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    count_le_kernel<<<static_cast<unsigned>(rows), 512, 0, st>>>(D, N, ldd, t, qnorm2, row_ids, self_col, out);
    return cudaGetLastError();
}

cudaError_t launch_band_count(const float* D, int64_t rows, int64_t N, int64_t ldd, const float* vals, int32_t k,
                              int32_t km, const float* E, const int32_t* self_col, const float* qnorm2,
                              const int32_t* row_ids, int32_t* out_count, int32_t* out_count4, float* out_edge,
                              cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    band_count_kernel<<<static_cast<unsigned>(rows), 512, 0, st>>>(D, N, ldd, vals, k, km, E, self_col, qnorm2,
                                                                   row_ids, out_count, out_count4, out_edge);
    return cudaGetLastError();
}

}  // namespace knn
