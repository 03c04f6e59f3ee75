// Cosine and Pearson similarity (Methods, "Distance calculation": the cosine metric
// x.y / (|x| |y|); the Pearson metric, the cosine of rows centred on their own mean).
//
// The k most similar points are found with the Euclidean engine: for unit vectors
// |u - v|^2 = 2 - 2 cos(u, v), so the nearest unit rows are the most similar rows.
//   1. sim_prep_kernel: per row, the FP64 mean (Pearson) and norm of the centred row,
//      and the unit row u = (x - mean) / norm rounded to FP32;
//   2. the Euclidean engine on the unit rows: the k' = k + m nearest (exact in the unit
//      rows' arithmetic);
//   3. sim_rerank_kernel: the similarity of every candidate from the original rows, its dot
//      product from FP32 error-free transformations (within 2^-38 of sum_t |a_t b_t|, see
//      pair_product_add), sorted by (similarity descending, index ascending); the k best are the
//      answer when the certificate below holds;
//   4. rows it does not certify are recomputed over the whole corpus in FP64.
//
// Certificate. Let s be the FP64 similarity computed from the same means and norms as
// the unit rows. Each unit entry carries a relative error of at most 2^-24 + 3 2^-53
// against (x - mean) / norm, which bounds |d2(u_i, u_j) - (2 - 2 s_ij)| by
// eta = 9 2^-24 + (4 d + 64) 2^-53. The re-rank's similarity is within 2^-38 (1 + 2^-40)
// of s (Cauchy-Schwarz: sum |a_t b_t| <= |a| |b|), so 2^-36 is added to the margin. The
// engine reports d2 of its k'-th candidate in FP32 (within 2^-18 of the value it ranked by),
// and every other point lies at least that far. So when
// 2 - 2 s_(k) < d2_(k') - 2^-18 - eta - 2^-36, no point outside the candidates can reach the
// k-th similarity, and the answer is exact.
#include "common.cuh"
#include "internal.h"

namespace knn {
namespace {

constexpr int RR_THREADS = 128;

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per row.
__global__ void sim_prep_kernel(const float* __restrict__ X, int64_t rows, int32_t d, int32_t centered,
                                float* __restrict__ U, double* __restrict__ mean, double* __restrict__ norm,
                                int32_t* __restrict__ bad) {
    const int64_t row = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (row >= rows) return;
    const int lane = static_cast<int>(threadIdx.x & 31u);
    const float* x = X + row * d;
    double m = 0.0;
    if (centered) {
        double s = 0.0;
        for (int t = lane; t < d; t += 32) s += static_cast<double>(x[t]);
        m = warp_sum_f64(s) / static_cast<double>(d);
    }
    double ss = 0.0;
    for (int t = lane; t < d; t += 32) {
        const double c = static_cast<double>(x[t]) - m;
        ss = fma(c, c, ss);
    }
    const double n = sqrt(warp_sum_f64(ss));
    const bool ok = n > 0.0 && n <= 1.7976931348623157e308;  // zero norm, NaN or Inf: undefined
    if (!ok) {
        if (lane == 0) atomicOr(bad, 1);
        return;
    }
    float* u = U + row * d;
    for (int t = lane; t < d; t += 32) u[t] = static_cast<float>((static_cast<double>(x[t]) - m) / n);
    if (lane == 0) {
        mean[row] = m;
        norm[row] = n;
    }
}

// a - m as an FP32 pair h + l within 2^-48 |a - m| of it, for an FP32 value a and an FP64
// mean m split as mh + ml (FP32 values, ml the rounding of m - mh): a - mh = s + e exactly
// and e - ml = e2 + r2 exactly (TwoSum, Knuth), s + e2 = h + l exactly, and r2, below 2^-24
// |e2|, is added to l with one rounding.
__device__ __forceinline__ void centre_pair(float a, float mh, float ml, float& h, float& l) {
    float s, e, e2, r2;
    two_sum(a, -mh, s, e);
    two_sum(e, -ml, e2, r2);
    two_sum(s, e2, h, l);
    l = __fadd_rn(l, r2);
}

// Dot-product accumulation of one lane, FP32 error-free transformations and an FP64 sum
// (pair_product_add, and the blocks of 8 in sim_rerank_kernel):
// the product of two pairs (ah + al)(bh + bl) is ah bh = p + pe exactly (the rounding error
// of the product recovered by an FMA, as in Dekker's and Ogita-Rump-Oishi's TwoProd), plus
// ah bl + al bh rounded into pe (al bl, below 2^-48 |ab|, dropped); the p's are summed by
// TwoSum into (S, E), and after every 8 terms S + E goes into the lane's FP64 sum. E holds
// the TwoSum errors and the pe's, at most 2^-19 of the block's sum |a_t b_t|; its own
// roundings stay below 2^-39 of it, so the lanes' total is within 2^-38 sum_t |a_t b_t|.
__device__ __forceinline__ void pair_product_add(float ah, float al, float bh, float bl, float& S, float& E) {
    const float pr = __fmul_rn(ah, bh);
    float pe = __fmaf_rn(ah, bh, -pr);
    pe = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, pe));
    float s2, e2;
    two_sum(S, pr, s2, e2);
    S = s2;
    E = __fadd_rn(E, __fadd_rn(e2, pe));
}

// One block per query row: similarity of the candidates, sort, certificate, output. The
// (centred) query row is staged in shared memory as FP32 pairs when it fits (STAGED). Each
// reported unit-row distance is within margin of 2 - 2 s, so the k nearest candidates all
// have s >= 1 - (d2_(k) + margin) / 2; a later candidate with d2 > d2_(k) + 2 margin has a
// smaller s than that and cannot enter the answer: its FP64 similarity is skipped.
template <bool CENTERED, bool STAGED>
__global__ void __launch_bounds__(RR_THREADS) sim_rerank_kernel(SimRerankParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* S = reinterpret_cast<double*>(smem_raw);
    int32_t* I = reinterpret_cast<int32_t*>(S + p.P);
    float2* Qs = reinterpret_cast<float2*>(I + p.P + (p.P & 1));
    const int64_t i = blockIdx.x;
    const int warp = static_cast<int>(threadIdx.x >> 5), lane = static_cast<int>(threadIdx.x & 31u);
    const int nw = RR_THREADS / 32;
    const float* q = p.Q + i * p.d;
    const double mi = CENTERED ? p.qmean[i] : 0.0;
    const float mih = static_cast<float>(mi), mil = static_cast<float>(mi - static_cast<double>(mih));
    const double ni = p.qnorm[i];
    if (STAGED) {
        for (int t = static_cast<int>(threadIdx.x); t < p.d; t += RR_THREADS) {
            float h = q[t], l = 0.f;
            if (CENTERED) centre_pair(q[t], mih, mil, h, l);
            Qs[t] = make_float2(h, l);
        }
        __syncthreads();
    }
    const double skip_above = static_cast<double>(p.cand_dist[i * p.kp + p.k - 1]) + 2.0 * p.margin;
    for (int c = warp; c < p.P; c += nw) {
        int32_t j = c < p.kp ? p.cand_idx[i * p.kp + c] : -1;
        if (j >= 0 && c >= p.k && static_cast<double>(p.cand_dist[i * p.kp + c]) > skip_above) j = -1;
        double s = -__longlong_as_double(0x7ff0000000000000ll);  // -inf: no candidate
        if (j >= 0) {
            const float* y = p.C + static_cast<int64_t>(j) * p.d;
            const double mj = CENTERED ? p.cmean[j] : 0.0;
            const float mjh = static_cast<float>(mj), mjl = static_cast<float>(mj - static_cast<double>(mjh));
            // the lane's elements t0 + 32 u (u < 8) form one block: loaded first (eight loads
            // in flight), then summed, then folded into the FP64 sum; a block past the end of
            // the row adds zeros, which change neither S nor E
            double acc = 0.0;
            for (int t0 = lane; t0 < p.d; t0 += 256) {
                float yv[8], qh[8], ql[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int t = t0 + 32 * u;
                    const bool in = t < p.d;
                    yv[u] = in ? y[t] : 0.f;
                    if (STAGED) {
                        const float2 a = in ? Qs[t] : make_float2(0.f, 0.f);
                        qh[u] = a.x;
                        ql[u] = a.y;
                    } else {
                        qh[u] = in ? q[t] : 0.f;
                        ql[u] = 0.f;
                    }
                }
                float S = 0.f, E = 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const bool in = t0 + 32 * u < p.d;
                    float ah = qh[u], al = ql[u], bh = yv[u], bl = 0.f;
                    if (CENTERED && in) {
                        if (!STAGED) centre_pair(qh[u], mih, mil, ah, al);
                        centre_pair(yv[u], mjh, mjl, bh, bl);
                    }
                    pair_product_add(ah, al, bh, bl, S, E);
                }
                acc += static_cast<double>(S) + static_cast<double>(E);
            }
            const double dot = warp_sum_f64(acc);
            s = dot / (ni * p.cnorm[j]);
        }
        if (lane == 0) {
            S[c] = s;
            I[c] = j >= 0 ? j : 0x7fffffff;
        }
    }
    __syncthreads();
    // bitonic sort by (similarity descending, index ascending)
    for (int size = 2; size <= p.P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = static_cast<int>(threadIdx.x); t < (p.P >> 1); t += RR_THREADS) {
                const int a = 2 * t - (t & (stride - 1));
                const int b = a + stride;
                const bool up = (a & size) == 0;
                const double sa = S[a], sb = S[b];
                const int32_t ia = I[a], ib = I[b];
                const bool a_after_b = sa < sb || (sa == sb && ia > ib);
                if (a_after_b == up) {
                    S[a] = sb;
                    S[b] = sa;
                    I[a] = ib;
                    I[b] = ia;
                }
            }
            __syncthreads();
        }
    for (int t = static_cast<int>(threadIdx.x); t < p.k; t += RR_THREADS) {
        p.out_idx[i * p.k + t] = I[t] == 0x7fffffff ? -1 : I[t];
        p.out_val[i * p.k + t] = static_cast<float>(S[t]);
    }
    if (threadIdx.x == 0) {
        bool cert = p.all_candidates != 0;
        if (!cert) {
            const double edge = static_cast<double>(p.cand_dist[i * p.kp + p.kp - 1]) - p.margin;
            cert = 2.0 - 2.0 * S[p.k - 1] < edge;
        }
        p.uncertified[i] = cert ? 0u : 1u;
    }
}

}  // namespace

cudaError_t launch_sim_prep(const float* X, int64_t rows, int32_t d, int32_t centered, float* U, double* mean,
                            double* norm, int32_t* bad, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (rows * 32 + threads - 1) / threads;
    sim_prep_kernel<<<static_cast<unsigned>(blocks), threads, 0, st>>>(X, rows, d, centered, U, mean, norm, bad);
    return cudaGetLastError();
}

double sim_margin(int32_t d) {
    // 2^-18 for the FP32 distance the engine reports, eta, and 2^-36 for the re-rank's
    // similarity (see the header comment)
    return 0x1p-18 + 9.0 * 0x1p-24 + (4.0 * d + 64.0) * 0x1p-53 + 0x1p-36;
}

cudaError_t launch_sim_rerank(const SimRerankParams& p, int32_t centered, cudaStream_t st) {
    if (p.M <= 0) return cudaSuccess;
    const size_t base = static_cast<size_t>(p.P) * (sizeof(double) + sizeof(int32_t)) + (p.P & 1) * sizeof(int32_t);
    const size_t staged = base + static_cast<size_t>(p.d) * sizeof(float2);
    const bool stage = staged <= 160 * 1024;
    const size_t smem = stage ? staged : base;
    auto kern = centered ? (stage ? sim_rerank_kernel<true, true> : sim_rerank_kernel<true, false>)
                         : (stage ? sim_rerank_kernel<false, true> : sim_rerank_kernel<false, false>);
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kern), static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(p.M), RR_THREADS, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace knn
