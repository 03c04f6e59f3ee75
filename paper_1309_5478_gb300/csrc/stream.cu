// Out-of-core corpus (the paper's Discussion: corpora beyond device memory): the corpus
// is searched chunk by chunk, and each chunk's exact answer is merged into the running
// answer of every query row by (FP64 direct-difference distance, global index) -- the order
// a search over the whole corpus gives.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace knn {
namespace {

constexpr int MG_THREADS = 128;

// One block per query row. The chunk's kc results (chunk-local indices) get their FP64
// direct-difference squared distances while the chunk is resident; with the running k
// entries they are sorted by (FP64 distance, global index) and the first k are kept, with
// the FP32 rounding of the FP64 distance as the reported value (a value of the pair alone,
// whatever the chunking).
template <bool STAGED>
__global__ void __launch_bounds__(MG_THREADS) stream_merge_kernel(StreamMergeParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* K = reinterpret_cast<double*>(smem_raw);     // P FP64 distances
    int64_t* J = reinterpret_cast<int64_t*>(K + p.P);    // P global indices
    double* Qs = reinterpret_cast<double*>(J + p.P);
    const int64_t i = blockIdx.x;
    const int warp = static_cast<int>(threadIdx.x >> 5), lane = static_cast<int>(threadIdx.x & 31u);
    const float* q = p.Q + i * p.d;
    if (STAGED) {
        for (int t = static_cast<int>(threadIdx.x); t < p.d; t += MG_THREADS) Qs[t] = static_cast<double>(q[t]);
    }
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    for (int t = static_cast<int>(threadIdx.x); t < p.P; t += MG_THREADS) {
        if (t < p.k) {
            K[t] = p.run_d64[i * p.k + t];
            J[t] = p.run_idx[i * p.k + t] < 0 ? INT64_MAX : static_cast<int64_t>(p.run_idx[i * p.k + t]);
        } else if (t >= p.k + p.kc) {
            K[t] = inf;
            J[t] = INT64_MAX;
        }
    }
    __syncthreads();
    for (int c = warp; c < p.kc; c += MG_THREADS / 32) {
        const int32_t j = p.chunk_idx[i * p.kc + c];
        double s = inf;
        if (j >= 0) {
            const float* y = p.chunk + static_cast<int64_t>(j) * p.d;
            double acc = 0.0;
            for (int t = lane; t < p.d; t += 32) {
                const double diff = (STAGED ? Qs[t] : static_cast<double>(q[t])) - static_cast<double>(y[t]);
                acc = fma(diff, diff, acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            s = acc;
        }
        if (lane == 0) {
            K[p.k + c] = s;
            J[p.k + c] = j >= 0 ? p.chunk_row0 + j : INT64_MAX;
        }
    }
    __syncthreads();
    for (int size = 2; size <= p.P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = static_cast<int>(threadIdx.x); t < (p.P >> 1); t += MG_THREADS) {
                const int a = 2 * t - (t & (stride - 1));
                const int b = a + stride;
                const bool up = (a & size) == 0;
                const double ka = K[a], kb = K[b];
                const int64_t ja = J[a], jb = J[b];
                const bool a_after_b = ka > kb || (ka == kb && ja > jb);
                if (a_after_b == up) {
                    K[a] = kb;
                    K[b] = ka;
                    J[a] = jb;
                    J[b] = ja;
                }
            }
            __syncthreads();
        }
    for (int t = static_cast<int>(threadIdx.x); t < p.k; t += MG_THREADS) {
        p.run_d64[i * p.k + t] = K[t];
        p.run_idx[i * p.k + t] = J[t] == INT64_MAX ? -1 : static_cast<int32_t>(J[t]);
        p.run_f32[i * p.k + t] = static_cast<float>(K[t]);
    }
}

// A later chunk's point enters query i's answer only when its distance is below the running
// k-th (one at the same distance has a higher index and loses the tie), so the running k-th,
// rounded up, bounds what the next chunk's search has to find.
__global__ void stream_bound_kernel(const double* __restrict__ run_d64, int64_t M, int32_t k,
                                    float* __restrict__ thr) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const double v = run_d64[i * k + k - 1];
    float f = static_cast<float>(v);
    if (static_cast<double>(f) < v) f = nextafterf(f, __int_as_float(0x7f800000));
    thr[i] = f;
}

__global__ void stream_init_kernel(int64_t n, int32_t* idx, double* d64, float* f32) {
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        idx[t] = -1;
        d64[t] = __longlong_as_double(0x7ff0000000000000ll);
        f32[t] = __int_as_float(0x7f800000);
    }
}

}  // namespace

cudaError_t launch_stream_init(int64_t n, int32_t* idx, double* d64, float* f32, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    stream_init_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(n, idx, d64, f32);
    return cudaGetLastError();
}

cudaError_t launch_stream_bound(const double* run_d64, int64_t M, int32_t k, float* thr, cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    stream_bound_kernel<<<static_cast<unsigned>((M + 255) / 256), 256, 0, st>>>(run_d64, M, k, thr);
    return cudaGetLastError();
}

cudaError_t launch_stream_merge(const StreamMergeParams& p, cudaStream_t st) {
    if (p.M <= 0) return cudaSuccess;
    const size_t base = static_cast<size_t>(p.P) * (sizeof(double) + sizeof(int64_t));
    const size_t staged = base + static_cast<size_t>(p.d) * sizeof(double);
    const bool stage = staged <= 160 * 1024;
    const size_t smem = stage ? staged : base;
    auto kern = stage ? stream_merge_kernel<true> : stream_merge_kernel<false>;
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kern), static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(p.M), MG_THREADS, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace knn
