// FP32 SIMT distance GEMM (the plain form).
//
// Paper: Methods, "Distance calculation": the n x m dot products x_i.y_j are the
// matrix product X^T Y, and the k nearest of x_i can be ranked by
// d'_ij = |y_j|^2 - 2 x_i.y_j because |x_i|^2 is common to the whole row. This
// kernel writes d' (or d2 = |x_i|^2 + d') for a slab of query rows against all
// corpus points, i.e. it materialises the distance matrix that the unfused
// quick multi-select then reads.
//
// Both operands are row-major with the shared dimension d contiguous ("K-major").
// Tiling: 128 x 128 output tile per 256-thread block, 8 x 8 outputs per thread (a 64 x 128
// tile with 4 x 8 outputs a thread for at most 64 query rows, the band probe's sample),
// k-slices of 16 staged in shared memory (transposed so threads read contiguous
// rows of the tile), double-buffered with register prefetch. Each output is one FMA
// chain over t = 0..d-1, so its rounding error is bounded by gamma_d |q||c|.
#include "common.cuh"
#include "internal.h"

namespace knn {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, TN = 8, NT = 256;
constexpr int LDS = BM + 4;  // padded shared-memory row

// Loads H halves of 64 rows of a BK-wide k-slice (H = 2: a 128-row tile).
template <bool VEC, int H = 2>
__device__ __forceinline__ void load_tile(const float* __restrict__ X, int64_t rows, int64_t r0, int32_t d, int k0,
                                          float (&reg)[2][4]) {
    // thread t loads rows (t/4) and (t/4 + 64), k-quad (t % 4)
    const int lr = static_cast<int>(threadIdx.x) / 4;
    const int lk = (static_cast<int>(threadIdx.x) % 4) * 4;
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int64_t r = r0 + lr + h * 64;
        const int kk = k0 + lk;
        if (VEC) {
            if (r < rows && kk + 3 < d) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(X + r * d + kk));
                reg[h][0] = v.x;
                reg[h][1] = v.y;
                reg[h][2] = v.z;
                reg[h][3] = v.w;
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) reg[h][c] = (r < rows && kk + c < d) ? X[r * d + kk + c] : 0.f;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) reg[h][c] = (r < rows && kk + c < d) ? X[r * d + kk + c] : 0.f;
        }
    }
}

template <int H = 2>
__device__ __forceinline__ void store_tile(float (*S)[LDS], const float (&reg)[2][4]) {
    const int lr = static_cast<int>(threadIdx.x) / 4;
    const int lk = (static_cast<int>(threadIdx.x) % 4) * 4;
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
        for (int c = 0; c < 4; ++c) S[lk + c][lr + h * 64] = reg[h][c];
}

// QH: 64-row halves of the query tile (2: 128 x 128 tiles, 8 x 8 outputs a thread; 1: 64 x 128,
// 4 x 8 outputs a thread).
template <bool VEC, int QH>
__global__ void __launch_bounds__(NT) gemm_dprime_kernel(const float* __restrict__ Q, int64_t M, int64_t row0,
                                                          const float* __restrict__ C, int64_t N, int32_t d,
                                                          const float* __restrict__ cnorm2,
                                                          const float* __restrict__ qnorm2, float* __restrict__ D,
                                                          int64_t ldd, int32_t exclude_self) {
    __shared__ __align__(16) float As[2][BK][LDS];
    __shared__ __align__(16) float Bs[2][BK][LDS];
    constexpr int TM = 4 * QH;
    const int64_t m0 = static_cast<int64_t>(blockIdx.y) * (64 * QH);
    const int64_t n0 = static_cast<int64_t>(blockIdx.x) * BN;
    const int tx = static_cast<int>(threadIdx.x) % 16;
    const int ty = static_cast<int>(threadIdx.x) / 16;

    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

    float ra[2][4], rb[2][4];
    load_tile<VEC, QH>(Q, M, m0, d, 0, ra);
    load_tile<VEC>(C, N, n0, d, 0, rb);
    store_tile<QH>(As[0], ra);
    store_tile(Bs[0], rb);
    __syncthreads();

    const int ktiles = (d + BK - 1) / BK;
    for (int kt = 0; kt < ktiles; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < ktiles) {
            load_tile<VEC, QH>(Q, M, m0, d, (kt + 1) * BK, ra);
            load_tile<VEC>(C, N, n0, d, (kt + 1) * BK, rb);
        }
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
            const float4 a1 = QH == 2 ? *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]) : a0;
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < ktiles) {
            store_tile<QH>(As[cur ^ 1], ra);
            store_tile(Bs[cur ^ 1], rb);
        }
        __syncthreads();
    }

    // epilogue: d' = |c|^2 - 2 q.c  (+ |q|^2)
    const bool vec_out = (ldd % 4) == 0;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (r >= M) continue;
        const float qa = qnorm2 ? qnorm2[r] : 0.f;
        float* drow = D + r * ldd;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t c0 = n0 + h * 64 + tx * 4;
            float v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t c = c0 + j;
                const float cn = c < N ? cnorm2[c] : 0.f;
                float x = fmaf(-2.f, acc[i][h * 4 + j], cn) + qa;
                if (exclude_self && row0 + r == c) x = F_INF;
                v[j] = x;
            }
            if (vec_out && c0 + 3 < N) {
                *reinterpret_cast<float4*>(drow + c0) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (c0 + j < N) drow[c0 + j] = v[j];
            }
        }
    }
}

}  // namespace

cudaError_t launch_gemm_simt(const float* Q, int64_t M, int64_t row0, const float* C, int64_t N, int32_t d,
                             const float* cnorm2, const float* qnorm2, float* D, int64_t ldd, int32_t exclude_self,
                             cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    // at most 64 query rows (the band probe's sample): 64-row tiles, no half-empty tile
    const bool skinny = M <= 64;
    const dim3 grid(static_cast<unsigned>((N + BN - 1) / BN),
                    static_cast<unsigned>(skinny ? 1 : (M + BM - 1) / BM));
    const bool vec = (d % 4 == 0) && (reinterpret_cast<uintptr_t>(Q) % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(C) % 16 == 0) && (reinterpret_cast<uintptr_t>(D) % 16 == 0);
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    if (skinny) {
        if (vec)
            gemm_dprime_kernel<true, 1><<<grid, NT, 0, st>>>(Q, M, row0, C, N, d, cnorm2, qnorm2, D, ldd, exclude_self);
        else
            gemm_dprime_kernel<false, 1><<<grid, NT, 0, st>>>(Q, M, row0, C, N, d, cnorm2, qnorm2, D, ldd, exclude_self);
    } else if (vec) {
        gemm_dprime_kernel<true, 2><<<grid, NT, 0, st>>>(Q, M, row0, C, N, d, cnorm2, qnorm2, D, ldd, exclude_self);
    } else {
        gemm_dprime_kernel<false, 2><<<grid, NT, 0, st>>>(Q, M, row0, C, N, d, cnorm2, qnorm2, D, ldd, exclude_self);
    }
    return cudaGetLastError();
}

}  // namespace knn
