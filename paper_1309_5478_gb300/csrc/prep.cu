// Pre-processing: per-row squared norms and the reduced-precision copies of the
// points, plus the per-row error bounds used to keep reduced-precision selection
// exact.
//
// Paper: Methods, "Distance calculation" -- the squared norms |x|^2 are vector
// reductions computed before the distance product (there with a transform
// iterator feeding reduction_by_key). Here one warp reduces one row and the
// same pass writes the BF16 / FP8 copy consumed by the tensor-core GEMM.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "internal.h"

namespace knn {
namespace {

__device__ __forceinline__ void atomic_max_bits(uint32_t* p, float v) {
    // v >= 0: the bit pattern's unsigned order is the value order
    atomicMax(p, __float_as_uint(v));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Reduced-precision rounding of one value: returns the rounded value as FP32 and
// stores its encoding.
template <int P>
__device__ __forceinline__ float quantise(float x, float scale, void* xq, int64_t off) {
    if constexpr (P == P_BF16) {
        __nv_bfloat16 h = __float2bfloat16_rn(x);
        static_cast<__nv_bfloat16*>(xq)[off] = h;
        return __bfloat162float(h);
    } else if constexpr (P == P_FP8) {
        __nv_fp8_e4m3 q(x * scale);  // saturating round-to-nearest-even
        static_cast<__nv_fp8_e4m3*>(xq)[off] = q;
        return static_cast<float>(q) / scale;  // scale is a power of two: exact
    } else {
        return x;
    }
}

// Statistics of the rows a warp has prepared, flushed to a problem's PrepGlobals with one
// set of atomics (values >= 0 compare as their bit patterns).
struct RowStatsAcc {
    float max_res = 0.f, max_tnorm = 0.f, max_norm2 = 0.f, max_abs = 0.f;
    uint32_t nonfinite = 0, noninteger = 0;
    __device__ __forceinline__ void flush(PrepGlobals* g, bool reduced) {
        if (lane_id() != 0) return;
        if (reduced) {
            atomic_max_bits(&g->max_res, max_res);
            atomic_max_bits(&g->max_tnorm, max_tnorm);
        }
        atomic_max_bits(&g->max_norm2, max_norm2);
        atomic_max_bits(&g->max_abs, max_abs);
        if (nonfinite) atomicAdd(&g->nonfinite, nonfinite);
        if (noninteger) atomicAdd(&g->noninteger, noninteger);
        *this = RowStatsAcc{};
    }
};

// One warp prepares one row: norms, the reduced-precision copy, and the row's statistics
// into acc (every lane holds the same values).
template <int P>
__device__ __forceinline__ void prep_row(const float* __restrict__ X, int64_t row, int32_t d,
                                         float* __restrict__ norm2, float* __restrict__ res,
                                         float* __restrict__ tnorm, void* __restrict__ xq, int32_t ldq,
                                         float* __restrict__ inv_scale, RowStatsAcc& acc) {
    const uint32_t lane = lane_id();
    const float* x = X + row * static_cast<int64_t>(d);

    float s2 = 0.f, amax = 0.f;
    bool bad = false, nonint = false;
    for (int32_t t = lane; t < d; t += 32) {
        float v = x[t];
        s2 = fmaf(v, v, s2);
        amax = fmaxf(amax, fabsf(v));
        bad |= !isfinite(v);
        nonint |= (v != rintf(v));
    }
    s2 = warp_sum(s2);
    amax = warp_maxf(amax);
    bad = __any_sync(0xffffffffu, bad);
    nonint = __any_sync(0xffffffffu, nonint);

    float scale = 1.f;
    if constexpr (P == P_FP8) {
        // power-of-two scale putting the row's largest magnitude in (224, 448]
        int e = 0;
        if (amax > 0.f && isfinite(amax)) {
            frexpf(amax / 448.f, &e);  // amax / 448 = m * 2^e, m in [0.5, 1)
            e = -e;                    // amax * 2^-e... -> amax * 2^e in (224, 448]
        }
        scale = ldexpf(1.f, e);
    }

    if constexpr (P != P_FP32) {
        float r2 = 0.f, t2 = 0.f;
        const int64_t base = row * static_cast<int64_t>(ldq);
        for (int32_t t = lane; t < ldq; t += 32) {
            float v = t < d ? x[t] : 0.f;
            float vq = quantise<P>(v, scale, xq, base + t);
            float r = v - vq;  // exact: vq is v rounded to fewer bits
            r2 = fmaf(r, r, r2);
            t2 = fmaf(vq, vq, t2);
        }
        r2 = warp_sum(r2);
        t2 = warp_sum(t2);
        // upper bounds on the norms (FP32 sum and sqrt rounding absorbed by the factor)
        const float inflate = 1.f + 0x1p-12f;
        float rn = sqrtf(r2) * inflate, tn = sqrtf(t2) * inflate;
        if (lane == 0) {
            res[row] = rn;
            tnorm[row] = tn;
            if (inv_scale) inv_scale[row] = 1.f / scale;
        }
        acc.max_res = fmaxf(acc.max_res, rn);
        acc.max_tnorm = fmaxf(acc.max_tnorm, tn);
    }
    if (lane == 0) norm2[row] = s2;
    if (!bad) {
        acc.max_norm2 = fmaxf(acc.max_norm2, s2);
        acc.max_abs = fmaxf(acc.max_abs, amax);
    }
    acc.nonfinite += bad ? 1u : 0u;
    acc.noninteger += nonint ? 1u : 0u;
}

constexpr int PREP_ROWS_PER_WARP = 16;

// prep_row for rows of 16-byte aligned groups of four (d % 4 == 0, aligned X): 16-byte
// loads and packed stores of the reduced-precision copy (8 bytes of BF16 or 4 of FP8 per
// lane and group). BF16 needs no row scale, so one pass reads the row once; FP8 first
// finds the row's largest magnitude. Same values and statistics as prep_row (sums in
// another order).
template <int P>
__device__ __forceinline__ void prep_row_vec(const float* __restrict__ X, int64_t row, int32_t d,
                                             float* __restrict__ norm2, float* __restrict__ res,
                                             float* __restrict__ tnorm, void* __restrict__ xq, int32_t ldq,
                                             float* __restrict__ inv_scale, RowStatsAcc& acc) {
    const uint32_t lane = lane_id();
    const float4* x4 = reinterpret_cast<const float4*>(X + row * static_cast<int64_t>(d));
    const int32_t g = d / 4;                              // groups of the row
    const int32_t gq = P == P_FP32 ? g : ldq / 4;         // groups of the padded copy
    float s2 = 0.f, amax = 0.f, r2 = 0.f, t2 = 0.f;
    bool bad = false, nonint = false;
    auto stats = [&](const float4 v) {
        const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            s2 = fmaf(e[c], e[c], s2);
            amax = fmaxf(amax, fabsf(e[c]));
            bad |= !isfinite(e[c]);
            nonint |= (e[c] != rintf(e[c]));
        }
    };
    if constexpr (P == P_BF16) {
        uint2* out = reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(xq) + row * static_cast<int64_t>(ldq));
        for (int32_t t = lane; t < gq; t += 32) {
            const float4 v = t < g ? __ldg(x4 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
            stats(v);
            const float e[4] = {v.x, v.y, v.z, v.w};
            uint32_t h[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const __nv_bfloat16 b = __float2bfloat16_rn(e[c]);
                const float vq = __bfloat162float(b);
                const float r = e[c] - vq;  // exact: vq is e rounded to fewer bits
                r2 = fmaf(r, r, r2);
                t2 = fmaf(vq, vq, t2);
                h[c] = __bfloat16_as_ushort(b);
            }
            out[t] = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
        }
    } else {
        for (int32_t t = lane; t < g; t += 32) stats(__ldg(x4 + t));
    }
    s2 = warp_sum(s2);
    amax = warp_maxf(amax);
    bad = __any_sync(0xffffffffu, bad);
    nonint = __any_sync(0xffffffffu, nonint);
    float scale = 1.f;
    if constexpr (P == P_FP8) {
        // power-of-two scale putting the row's largest magnitude in (224, 448]
        int e = 0;
        if (amax > 0.f && isfinite(amax)) {
            frexpf(amax / 448.f, &e);
            e = -e;
        }
        scale = ldexpf(1.f, e);
        uint32_t* out = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(xq) + row * static_cast<int64_t>(ldq));
        for (int32_t t = lane; t < gq; t += 32) {
            const float4 v = t < g ? __ldg(x4 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float e4[4] = {v.x, v.y, v.z, v.w};
            uint32_t word = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const __nv_fp8_e4m3 q(e4[c] * scale);  // saturating round-to-nearest-even
                const float vq = static_cast<float>(q) / scale;  // scale is a power of two: exact
                const float r = e4[c] - vq;
                r2 = fmaf(r, r, r2);
                t2 = fmaf(vq, vq, t2);
                word |= static_cast<uint32_t>(q.__x) << (8 * c);
            }
            out[t] = word;
        }
    }
    if constexpr (P != P_FP32) {
        r2 = warp_sum(r2);
        t2 = warp_sum(t2);
        // upper bounds on the norms (FP32 sum and sqrt rounding absorbed by the factor)
        const float inflate = 1.f + 0x1p-12f;
        const float rn = sqrtf(r2) * inflate, tn = sqrtf(t2) * inflate;
        if (lane == 0) {
            res[row] = rn;
            tnorm[row] = tn;
            if (inv_scale) inv_scale[row] = 1.f / scale;
        }
        acc.max_res = fmaxf(acc.max_res, rn);
        acc.max_tnorm = fmaxf(acc.max_tnorm, tn);
    }
    if (lane == 0) norm2[row] = s2;
    if (!bad) {
        acc.max_norm2 = fmaxf(acc.max_norm2, s2);
        acc.max_abs = fmaxf(acc.max_abs, amax);
    }
    acc.nonfinite += bad ? 1u : 0u;
    acc.noninteger += nonint ? 1u : 0u;
}

template <int P, bool VEC>
__global__ void __launch_bounds__(256) prep_kernel(const float* __restrict__ X, int64_t rows, int32_t d,
                                                   float* __restrict__ norm2, float* __restrict__ res,
                                                   float* __restrict__ tnorm, void* __restrict__ xq, int32_t ldq,
                                                   float* __restrict__ inv_scale, PrepGlobals* __restrict__ g) {
    const int64_t r0 = (static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32) * PREP_ROWS_PER_WARP;
    if (r0 >= rows) return;
    const int64_t r1 = r0 + PREP_ROWS_PER_WARP < rows ? r0 + PREP_ROWS_PER_WARP : rows;
    RowStatsAcc acc;
    for (int64_t row = r0; row < r1; ++row) {
        if constexpr (VEC)
            prep_row_vec<P>(X, row, d, norm2, res, tnorm, xq, ldq, inv_scale, acc);
        else
            prep_row<P>(X, row, d, norm2, res, tnorm, xq, ldq, inv_scale, acc);
    }
    acc.flush(g, P != P_FP32);
}

// Segment holding global row `row` (segs sorted by row0, segs[0].row0 == 0).
__device__ __forceinline__ int find_seg(const BatchSeg* segs, int32_t nseg, int64_t row) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].row0 <= row) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void batch_init_kernel(const BatchDev* __restrict__ probs, int32_t n) {
    const int32_t i = blockIdx.x;
    if (i >= n) return;
    const BatchDev& b = probs[i];
    constexpr int W = static_cast<int>(sizeof(PrepGlobals) / 4);
    if (threadIdx.x < W) {
        reinterpret_cast<uint32_t*>(b.gq)[threadIdx.x] = 0u;
        if (b.gc != b.gq) reinterpret_cast<uint32_t*>(b.gc)[threadIdx.x] = 0u;
    }
    if (b.xc) {
        const int64_t n_pad = (b.N + 255) / 256 * 256;
        for (int64_t j = b.N + threadIdx.x; j < n_pad; j += blockDim.x) b.cnorm2[j] = __uint_as_float(0xffffffffu);
    }
}

template <int P>
__global__ void __launch_bounds__(256) prep_batched_kernel(const BatchDev* __restrict__ probs,
                                                           const BatchSeg* __restrict__ segs, int32_t nseg,
                                                           int64_t rows) {
    const int64_t r0 = (static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32) * PREP_ROWS_PER_WARP;
    if (r0 >= rows) return;
    const int64_t r1 = r0 + PREP_ROWS_PER_WARP < rows ? r0 + PREP_ROWS_PER_WARP : rows;
    // a warp's rows span at most a few segments: the statistics are flushed per segment
    int64_t row = r0;
    while (row < r1) {
        const int si = find_seg(segs, nseg, row);
        const BatchSeg sg = segs[si];
        const int64_t seg_end = si + 1 < nseg ? segs[si + 1].row0 : rows;
        const int64_t stop = seg_end < r1 ? seg_end : r1;
        const BatchDev& b = probs[sg.problem];
        RowStatsAcc acc;
        // rows of four-value groups from 16-byte aligned bases take the 16-byte loads (the
        // reduced-precision copies are 256-byte aligned with rows of a multiple of 64 values)
        if (sg.which == 0) {
            for (; row < stop; ++row) {
                if (b.vec)
                    prep_row_vec<P>(b.C, row - sg.row0, b.d, b.cnorm2, b.cres, b.ctn, b.xc, b.d_pad, b.cscale, acc);
                else
                    prep_row<P>(b.C, row - sg.row0, b.d, b.cnorm2, b.cres, b.ctn, b.xc, b.d_pad, b.cscale, acc);
            }
            acc.flush(b.gc, P != P_FP32);
        } else {
            for (; row < stop; ++row) {
                if (b.vec)
                    prep_row_vec<P>(b.Q, row - sg.row0, b.d, b.qnorm2, b.qres, b.qtn, b.xq, b.d_pad, b.qscale, acc);
                else
                    prep_row<P>(b.Q, row - sg.row0, b.d, b.qnorm2, b.qres, b.qtn, b.xq, b.d_pad, b.qscale, acc);
            }
            acc.flush(b.gq, P != P_FP32);
        }
    }
}

// Error bound of the ranking value d'_ij = |c_j|^2 - 2 q_i.c_j as computed by the
// engine, against its exact value, for every j of row i.
//   FP32:  an FMA chain over d products has |err| <= gamma_d sum|q_t c_t| <= gamma_d |q||c|
//          (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.1); the norm
//          |c|^2 has gamma_d |c|^2 and the final FMA one more rounding. With
//          gamma_d <= (d + 2) 2^-24 and a factor 2 of safety:
//          E_i = (d + 4) 2^-23 (Cmax^2 + 2 |q_i| Cmax).
//   BF16 / FP8: with x = x~ + r (x~ the rounded copy), Cauchy-Schwarz gives
//          |q.c - q~.c~| <= |q~||r_c| + |r_q||c~| + |r_q||r_c|, doubled for the -2 q.c term;
//          the tensor-core FP32 accumulation is bounded like the FMA chain above
//          (safety factor 4 over FP32's gamma for BF16, a 2^-14-unit accumulator for FP8).
//   Exact arithmetic: integer-valued inputs with 4 d A^2 <= 2^24 (A the largest magnitude)
//          make every product, partial sum and norm an exact FP32 integer, so E_i = 0.
//   sym_extra (symmetric graph form): a transposed key is formed as (v - |x_j|^2) + |x_i|^2
//          from the value v of the other row, two more roundings of quantities at most
//          3 max|x|^2 in magnitude, covered by 2^-20 max|x|^2.
__device__ __forceinline__ void bounds_row(const float* __restrict__ qnorm2, const float* __restrict__ qres,
                                           const float* __restrict__ qtnorm, int64_t i, int32_t d, int32_t d_pad,
                                           int32_t precision, const PrepGlobals* __restrict__ gq,
                                           const PrepGlobals* __restrict__ gc, float* __restrict__ E,
                                           bool sym_extra = false) {
    const float amax = fmaxf(__uint_as_float(gq->max_abs), __uint_as_float(gc->max_abs));
    const bool integer = gq->noninteger == 0 && gc->noninteger == 0;
    const bool small = 4.0 * static_cast<double>(d_pad) * amax * amax <= 16777216.0;
    const bool rep = precision == P_FP32 || (precision == P_BF16 && amax <= 256.f) ||
                     (precision == P_FP8 && amax <= 16.f);
    if (integer && small && rep) {
        E[i] = 0.f;
        return;
    }
    const float c2max = __uint_as_float(gc->max_norm2);
    const float cmax = sqrtf(c2max) * (1.f + 0x1p-12f);
    const float qn = sqrtf(qnorm2[i]) * (1.f + 0x1p-12f);
    float e;
    if (precision == P_FP32) {
        e = static_cast<float>(d + 4) * 0x1p-23f * (c2max + 2.f * qn * cmax);
    } else {
        const float rmax = __uint_as_float(gc->max_res);
        const float ctmax = __uint_as_float(gc->max_tnorm);
        const float rq = qres[i], qt = qtnorm[i];
        const float quant = 2.f * (qt * rmax + rq * (ctmax + rmax));
        const float acc_unit = precision == P_BF16 ? 0x1p-22f : 0x1p-14f;
        const float accum = static_cast<float>(d_pad + 4) * acc_unit * 2.f * qt * ctmax;
        const float norms = static_cast<float>(d + 4) * 0x1p-23f * (c2max + 2.f * qn * cmax);
        e = quant + accum + norms;
    }
    if (sym_extra) e += 0x1p-20f * c2max;
    E[i] = e * (1.f + 0x1p-10f);
}

__global__ void bounds_kernel(const float* __restrict__ qnorm2, const float* __restrict__ qres,
                              const float* __restrict__ qtnorm, int64_t M, int32_t d, int32_t d_pad,
                              int32_t precision, const PrepGlobals* __restrict__ gq,
                              const PrepGlobals* __restrict__ gc, float* __restrict__ E, bool sym_extra) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= M) return;
    bounds_row(qnorm2, qres, qtnorm, i, d, d_pad, precision, gq, gc, E, sym_extra);
}

__global__ void bounds_batched_kernel(const BatchDev* __restrict__ probs, const BatchSeg* __restrict__ segs,
                                      int32_t nseg, int64_t rows, int32_t precision) {
    const int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    const BatchSeg sg = segs[find_seg(segs, nseg, row)];
    const BatchDev& b = probs[sg.problem];
    const int64_t i = row - sg.row0;
    bounds_row(b.qnorm2, b.qres, b.qtn, i, b.d, b.d_pad, precision, b.gq, b.gc, b.E);
    if (b.E32 != b.E) bounds_row(b.qnorm2, nullptr, nullptr, i, b.d, b.d, P_FP32, b.gq, b.gc, b.E32);
}

__global__ void thr_kernel(const float* __restrict__ thr, const float* __restrict__ qnorm2, int64_t M,
                           float* __restrict__ out) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const float t = thr[i];
    // non-finite or negative proposals mean "no threshold" for that row
    out[i] = (t == t && t >= 0.f && t < F_INF) ? t - qnorm2[i] : F_INF;
}

// A bounding threshold t (squared distance) in the scale of the approximate values: a point with
// exact squared distance d2 <= t has exact d' = d2 - |q|^2 <= t - |q|^2 and approximate value at
// most that plus E. |q|^2 comes from the prep pass (an FP32 FMA chain per lane, then a five-level
// warp sum: relative error below (d / 32 + 6) 2^-24), so less than qnorm2 is subtracted by a
// margin of that size; the sum is formed in FP64 and rounded up to FP32.
__global__ void bound_kernel(const float* __restrict__ thr, const float* __restrict__ qnorm2,
                             const float* __restrict__ E, int64_t M, int32_t d, float* __restrict__ out) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const float t = thr[i];
    if (!(t == t && t >= 0.f && t < F_INF)) {
        out[i] = F_INF;
        return;
    }
    const double g = (static_cast<double>(d) / 32.0 + 8.0) * 0x1p-24;
    const double q2 = static_cast<double>(qnorm2[i]);
    const double e = E ? static_cast<double>(E[i]) : 0.0;
    const double v = static_cast<double>(t) * (1.0 + 0x1p-40) - q2 * (1.0 - g) + e * (1.0 + 0x1p-10);
    float f = static_cast<float>(v);
    if (static_cast<double>(f) < v) f = nextafterf(f, F_INF);
    out[i] = f;
}

__global__ void gather_rows_kernel(const float* __restrict__ Q, int32_t d, const int32_t* __restrict__ rows,
                                   int32_t n, const float* __restrict__ E, const float* __restrict__ thr,
                                   float* __restrict__ Qs, float* __restrict__ Es, float* __restrict__ Ts) {
    const int32_t i = blockIdx.x;
    if (i >= n) return;
    const int64_t r = rows[i];
    for (int32_t t = threadIdx.x; t < d; t += blockDim.x) Qs[static_cast<int64_t>(i) * d + t] = Q[r * d + t];
    if (threadIdx.x == 0) {
        Es[i] = E[r];
        if (thr) Ts[i] = thr[r];
    }
}

// Rows of a reduced-precision operand (row_bytes a multiple of 16) and their scales.
__global__ void gather_qrows_kernel(const uint4* __restrict__ xq, int32_t row_vec, const float* __restrict__ qscale,
                                    const int32_t* __restrict__ rows, int32_t n, uint4* __restrict__ out,
                                    float* __restrict__ out_scale) {
    const int32_t i = blockIdx.x;
    if (i >= n) return;
    const int64_t r = rows[i];
    for (int32_t t = threadIdx.x; t < row_vec; t += blockDim.x)
        out[static_cast<int64_t>(i) * row_vec + t] = xq[r * row_vec + t];
    if (threadIdx.x == 0 && qscale) out_scale[i] = qscale[r];
}

__global__ void scatter_out_kernel(const int32_t* __restrict__ rows, int32_t n, int32_t k,
                                   const int32_t* __restrict__ oi_s, const float* __restrict__ od_s,
                                   int32_t* __restrict__ oi, float* __restrict__ od) {
    const int32_t i = blockIdx.x;
    if (i >= n) return;
    const int64_t r = rows[i];
    for (int32_t t = threadIdx.x; t < k; t += blockDim.x) {
        oi[r * k + t] = oi_s[static_cast<int64_t>(i) * k + t];
        od[r * k + t] = od_s[static_cast<int64_t>(i) * k + t];
    }
}

}  // namespace

cudaError_t launch_gather_rows(const float* Q, int32_t d, const int32_t* rows, int32_t n, const float* E,
                               const float* thr, float* Qs, float* Es, float* Ts, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    gather_rows_kernel<<<n, 128, 0, st>>>(Q, d, rows, n, E, thr, Qs, Es, Ts);
    return cudaGetLastError();
}

cudaError_t launch_gather_qrows(const void* xq, int32_t row_bytes, const float* qscale, const int32_t* rows, int32_t n,
                                void* out, float* out_scale, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (row_bytes % 16 != 0) return cudaErrorInvalidValue;
    gather_qrows_kernel<<<n, 128, 0, st>>>(static_cast<const uint4*>(xq), row_bytes / 16, qscale, rows, n,
                                           static_cast<uint4*>(out), out_scale);
    return cudaGetLastError();
}

cudaError_t launch_scatter_out(const int32_t* rows, int32_t n, int32_t k, const int32_t* oi_s, const float* od_s,
                               int32_t* oi, float* od, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    scatter_out_kernel<<<n, 128, 0, st>>>(rows, n, k, oi_s, od_s, oi, od);
    return cudaGetLastError();
}

cudaError_t launch_threshold_to_dprime(const float* thr, const float* qnorm2, int64_t M, float* out,
                                       cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    thr_kernel<<<static_cast<unsigned>((M + 255) / 256), 256, 0, st>>>(thr, qnorm2, M, out);
    return cudaGetLastError();
}

cudaError_t launch_bound_to_dprime(const float* thr, const float* qnorm2, const float* E, int64_t M, int32_t d,
                                   float* out, cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    bound_kernel<<<static_cast<unsigned>((M + 255) / 256), 256, 0, st>>>(thr, qnorm2, E, M, d, out);
    return cudaGetLastError();
}

cudaError_t launch_prep(const float* X, int64_t rows, int32_t d, int32_t precision, float* norm2, float* res,
                        float* tnorm, void* xq, int32_t ldq, float* inv_scale, PrepGlobals* g, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const int warps = 8;
    const unsigned blocks = static_cast<unsigned>((rows + warps * PREP_ROWS_PER_WARP - 1) / (warps * PREP_ROWS_PER_WARP));
    // 16-byte groups: rows of d % 4 == 0 floats from a 16-byte aligned base; the copy's rows
    // (ldq a multiple of 64 BF16 or 128 FP8 values) are aligned for the packed stores
    const bool vec = d % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0 &&
                     (precision == P_FP32 || (ldq % 4 == 0 && reinterpret_cast<uintptr_t>(xq) % 16 == 0));
#define KNN_PREP_LAUNCH(PP)                                                                                       \
    (vec ? prep_kernel<PP, true><<<blocks, warps * 32, 0, st>>>(X, rows, d, norm2, res, tnorm, xq, ldq, inv_scale, g) \
         : prep_kernel<PP, false><<<blocks, warps * 32, 0, st>>>(X, rows, d, norm2, res, tnorm, xq, ldq, inv_scale, g))
    switch (precision) {
        case P_FP32: KNN_PREP_LAUNCH(P_FP32); break;
        case P_BF16: KNN_PREP_LAUNCH(P_BF16); break;
        case P_FP8: KNN_PREP_LAUNCH(P_FP8); break;
        default: return cudaErrorInvalidValue;
    }
#undef KNN_PREP_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_batch_init(const BatchDev* probs, int32_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    batch_init_kernel<<<static_cast<unsigned>(n), 256, 0, st>>>(probs, n);
    return cudaGetLastError();
}

cudaError_t launch_prep_batched(const BatchDev* probs, const BatchSeg* segs, int32_t nseg, int64_t rows,
                                int32_t precision, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const unsigned blocks = static_cast<unsigned>((rows + 8 * PREP_ROWS_PER_WARP - 1) / (8 * PREP_ROWS_PER_WARP));
    switch (precision) {
        case P_FP32: prep_batched_kernel<P_FP32><<<blocks, 256, 0, st>>>(probs, segs, nseg, rows); break;
        case P_BF16: prep_batched_kernel<P_BF16><<<blocks, 256, 0, st>>>(probs, segs, nseg, rows); break;
        case P_FP8: prep_batched_kernel<P_FP8><<<blocks, 256, 0, st>>>(probs, segs, nseg, rows); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_bounds_batched(const BatchDev* probs, const BatchSeg* segs, int32_t nseg, int64_t rows,
                                  int32_t precision, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    bounds_batched_kernel<<<static_cast<unsigned>((rows + 255) / 256), 256, 0, st>>>(probs, segs, nseg, rows,
                                                                                     precision);
    return cudaGetLastError();
}

cudaError_t launch_bounds(const float* qnorm2, const float* qres, const float* qtnorm, int64_t M, int32_t d,
                          int32_t d_pad, int32_t precision, const PrepGlobals* gq, const PrepGlobals* gc, float* E,
                          cudaStream_t st, bool sym_extra) {
    if (M <= 0) return cudaSuccess;
    const unsigned blocks = static_cast<unsigned>((M + 255) / 256);
    bounds_kernel<<<blocks, 256, 0, st>>>(qnorm2, qres, qtnorm, M, d, d_pad, precision, gq, gc, E, sym_extra);
    return cudaGetLastError();
}

}  // namespace knn
