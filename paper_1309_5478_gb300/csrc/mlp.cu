// Learned per-row threshold: a small MLP that proposes, for each query row, the
// squared distance below which its k nearest neighbours lie. The proposal only
// pre-filters candidates (knn_options.row_threshold): rows where it cuts into the answer
// are recomputed without it, so results stay exact whatever the network predicts.
//
// Features of a row (KNN_MLP_FEATURES = 257): log |q|^2 and the sorted log squared
// distances to 256 corpus samples chosen by the caller. Network: 257 -> 128 (ReLU) -> 1,
// FP32, predicting t = log d2_(k) (the row's exact k-th squared distance) from the
// standardised features. The threshold proposed is exp(y + margin), margin being a
// high quantile of held-out residuals t - y.
//
// Parameter layout (one FP32 array of knn_mlp_param_count() entries):
//   W1[128][257] | b1[128] | W2[128] | b2 | mu[257] | sigma[257] | margin
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "engine.h"
#include "internal.h"
#include "knn.h"
#include "select_core.cuh"

namespace knn {
namespace {

constexpr int NF = KNN_MLP_FEATURES;
constexpr int NH = KNN_MLP_HIDDEN;
constexpr int NS = NF - 1;  // corpus samples per row
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NH * NF;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH;
constexpr int N_TRAIN = OFF_B2 + 1;  // trainable parameters
constexpr int OFF_MU = N_TRAIN;
constexpr int OFF_SIGMA = OFF_MU + NF;
constexpr int OFF_MARGIN = OFF_SIGMA + NF;
constexpr int N_PARAMS = OFF_MARGIN + 1;
constexpr int ROWS_PER_BLOCK = 32;
constexpr float LOG_FLOOR = -69.0f;  // log(1e-30): floor for zero distances

// features[row][0] = log |q|^2; features[row][1..256] = sorted log d2 to the samples
__global__ void features_finish_kernel(const float* __restrict__ D, int64_t M, const float* __restrict__ qnorm2,
                                       float* __restrict__ out) {
    __shared__ uint32_t buf[8][NS];
    const int warp = static_cast<int>(threadIdx.x / 32);
    const int64_t row = static_cast<int64_t>(blockIdx.x) * 8 + warp;
    if (row >= M) return;
    const uint32_t lane = lane_id();
    uint32_t* b = buf[warp];
    for (int i = static_cast<int>(lane); i < NS; i += 32) {
        const float v = fmaxf(D[row * NS + i], 0.f);  // expanded form can round below 0
        b[i] = __float_as_uint(v);                    // non-negative: bits order like values
    }
    __syncwarp();
    warp_bitonic_sort_smem(b, NS);
    float* o = out + row * NF;
    if (lane == 0) o[0] = fmaxf(logf(fmaxf(qnorm2[row], 0.f)), LOG_FLOOR);
    for (int i = static_cast<int>(lane); i < NS; i += 32) o[1 + i] = fmaxf(logf(__uint_as_float(b[i])), LOG_FLOOR);
}

// mu, sigma of every feature over n rows (one block per feature, FP64 sums)
__global__ void feature_stats_kernel(const float* __restrict__ X, int64_t n, float* __restrict__ params) {
    const int f = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double v = X[r * NF + f];
        s += v;
        s2 += v * v;
    }
    __shared__ double ws[32], ws2[32];
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ws[threadIdx.x / 32] = s;
        ws2[threadIdx.x / 32] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, a2 = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) {
            a += ws[w];
            a2 += ws2[w];
        }
        const double mu = a / static_cast<double>(n > 0 ? n : 1);
        const double var = a2 / static_cast<double>(n > 0 ? n : 1) - mu * mu;
        params[OFF_MU + f] = static_cast<float>(mu);
        params[OFF_SIGMA + f] = static_cast<float>(sqrt(var > 1e-12 ? var : 1e-12));
    }
}

// One block: ROWS_PER_BLOCK rows x NH threads (one per hidden unit). Forward pass,
// and with grad != nullptr the loss 1/n sum (y - t)^2 and its gradient (atomics).
// out_y (optional) receives the predictions.
template <bool GRAD>
__global__ void __launch_bounds__(NH) mlp_kernel(const float* __restrict__ X, const float* __restrict__ T, int64_t n,
                                                 int64_t n_norm, const float* __restrict__ params,
                                                 float* __restrict__ grad, double* __restrict__ loss,
                                                 float* __restrict__ out_y) {
    __shared__ float xs[ROWS_PER_BLOCK][NF + 1];
    __shared__ float part[NH / 32][ROWS_PER_BLOCK];
    __shared__ float ys[ROWS_PER_BLOCK];
    const int h = static_cast<int>(threadIdx.x);
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * ROWS_PER_BLOCK;
    const int nr = static_cast<int>(std::min<int64_t>(ROWS_PER_BLOCK, n - r0));
    // standardised features of the block's rows
    for (int i = h; i < ROWS_PER_BLOCK * NF; i += NH) {
        const int r = i / NF, f = i % NF;
        float v = 0.f;
        if (r < nr) v = (X[(r0 + r) * NF + f] - params[OFF_MU + f]) / params[OFF_SIGMA + f];
        xs[r][f] = v;
    }
    __syncthreads();
    float acc[ROWS_PER_BLOCK];
#pragma unroll
    for (int r = 0; r < ROWS_PER_BLOCK; ++r) acc[r] = params[OFF_B1 + h];
    const float* w1 = params + OFF_W1 + static_cast<int64_t>(h) * NF;
    for (int f = 0; f < NF; ++f) {
        const float w = w1[f];
#pragma unroll
        for (int r = 0; r < ROWS_PER_BLOCK; ++r) acc[r] = fmaf(w, xs[r][f], acc[r]);
    }
    const float w2 = params[OFF_W2 + h];
    // y_r = b2 + sum_h W2[h] relu(acc_h)
#pragma unroll
    for (int r = 0; r < ROWS_PER_BLOCK; ++r) {
        float c = w2 * fmaxf(acc[r], 0.f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((h & 31) == 0) part[h / 32][r] = c;
    }
    __syncthreads();
    if (h < ROWS_PER_BLOCK) {
        float y = params[OFF_B2];
        for (int w = 0; w < NH / 32; ++w) y += part[w][h];
        ys[h] = y;
        if (out_y && h < nr) out_y[r0 + h] = y;
    }
    __syncthreads();
    if constexpr (GRAD) {
        // dL/dy_r = 2 (y_r - t_r) / n_norm
        float dy[ROWS_PER_BLOCK];
        double lsum = 0.0;
#pragma unroll
        for (int r = 0; r < ROWS_PER_BLOCK; ++r) {
            const float e = r < nr ? ys[r] - T[r0 + r] : 0.f;
            dy[r] = 2.f * e / static_cast<float>(n_norm);
            lsum += static_cast<double>(e) * e;
        }
        if (h == 0) {
            atomicAdd(loss, lsum / static_cast<double>(n_norm));
            float db2 = 0.f;
#pragma unroll
            for (int r = 0; r < ROWS_PER_BLOCK; ++r) db2 += dy[r];
            atomicAdd(&grad[OFF_B2], db2);
        }
        float dw2 = 0.f, db1 = 0.f;
        float dh[ROWS_PER_BLOCK];
#pragma unroll
        for (int r = 0; r < ROWS_PER_BLOCK; ++r) {
            const float a = fmaxf(acc[r], 0.f);
            dw2 = fmaf(dy[r], a, dw2);
            dh[r] = acc[r] > 0.f ? dy[r] * w2 : 0.f;
            db1 += dh[r];
        }
        atomicAdd(&grad[OFF_W2 + h], dw2);
        atomicAdd(&grad[OFF_B1 + h], db1);
        float* gw1 = grad + OFF_W1 + static_cast<int64_t>(h) * NF;
        for (int f = 0; f < NF; ++f) {
            float g = 0.f;
#pragma unroll
            for (int r = 0; r < ROWS_PER_BLOCK; ++r) g = fmaf(dh[r], xs[r][f], g);
            atomicAdd(&gw1[f], g);
        }
    }
}

__global__ void adam_kernel(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void threshold_kernel(const float* __restrict__ y, int64_t n, const float* __restrict__ params,
                                 float* __restrict__ out) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = expf(y[i] + params[OFF_MARGIN]);
}

}  // namespace
}  // namespace knn

using namespace knn;

extern "C" int32_t knn_mlp_param_count(void) { return N_PARAMS; }

extern "C" int knn_mlp_features(const float* Q, int64_t M, const float* S, int32_t d, float* out_features,
                                const knn_options* opt) {
    g_last_error.clear();
    if (!Q || !S || !out_features) return set_error(KNN_EINVAL, "NULL pointer argument");
    if (M < 0 || d < 1) return set_error(KNN_EINVAL, "bad sizes");
    if (!is_device_pointer(Q) || !is_device_pointer(S) || !is_device_pointer(out_features))
        return set_error(KNN_EINVAL, "knn_mlp_features takes device pointers");
    if (M == 0) return KNN_OK;
    cudaStream_t st = opt ? static_cast<cudaStream_t>(opt->stream) : nullptr;
    // slabs of query rows bound the distance workspace (slab x 256 floats)
    const int64_t slab = std::min<int64_t>(M, int64_t(1) << 16);
    Arena sz;
    sz.take<PrepGlobals>(2);
    sz.take<float>(NS);
    sz.take<float>(M);
    sz.take<float>(static_cast<size_t>(slab) * NS);
    void* base = nullptr;
    KNN_TRY(workspace_get(sz.used(), &base));
    Arena ar(static_cast<char*>(base), sz.used());
    PrepGlobals* g = ar.take<PrepGlobals>(2);
    float* sn = ar.take<float>(NS);
    float* qn = ar.take<float>(M);
    float* D = ar.take<float>(static_cast<size_t>(slab) * NS);
    KNN_CK(cudaMemsetAsync(g, 0, 2 * sizeof(PrepGlobals), st));
    KNN_CK(launch_prep(S, NS, d, P_FP32, sn, nullptr, nullptr, nullptr, 0, nullptr, g, st));
    KNN_CK(launch_prep(Q, M, d, P_FP32, qn, nullptr, nullptr, nullptr, 0, nullptr, g + 1, st));
    for (int64_t r0 = 0; r0 < M; r0 += slab) {
        const int64_t m = std::min<int64_t>(slab, M - r0);
        KNN_CK(launch_gemm_simt(Q + r0 * d, m, 0, S, NS, d, sn, qn + r0, D, NS, 0, st));
        features_finish_kernel<<<static_cast<unsigned>((m + 7) / 8), 256, 0, st>>>(D, m, qn + r0,
                                                                                   out_features + r0 * NF);
        KNN_CK(cudaGetLastError());
    }
    KNN_CK(cudaStreamSynchronize(st));
    return KNN_OK;
}

extern "C" int knn_mlp_loss_grad(const float* features, const float* targets, int64_t n, const float* params,
                                 double* out_loss, float* out_grad, const knn_options* opt) {
    g_last_error.clear();
    if (!features || !targets || !params || !out_loss || !out_grad) return set_error(KNN_EINVAL, "NULL pointer");
    if (n < 1) return set_error(KNN_EINVAL, "n must be >= 1");
    cudaStream_t st = opt ? static_cast<cudaStream_t>(opt->stream) : nullptr;
    Arena sz;
    sz.take<double>(1);
    void* base = nullptr;
    KNN_TRY(workspace_get(sz.used(), &base));
    Arena ar(static_cast<char*>(base), sz.used());
    double* loss = ar.take<double>(1);
    KNN_CK(cudaMemsetAsync(loss, 0, sizeof(double), st));
    KNN_CK(cudaMemsetAsync(out_grad, 0, N_TRAIN * sizeof(float), st));
    const unsigned blocks = static_cast<unsigned>((n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
    mlp_kernel<true><<<blocks, NH, 0, st>>>(features, targets, n, n, params, out_grad, loss, nullptr);
    KNN_CK(cudaGetLastError());
    KNN_CK(cudaMemcpyAsync(out_loss, loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaStreamSynchronize(st));
    return KNN_OK;
}

extern "C" int knn_mlp_train(const float* features, const float* targets, int64_t n, float* params, int32_t epochs,
                             int32_t batch, float lr, float holdout, float margin_quantile, float* out_history,
                             const knn_options* opt) {
    g_last_error.clear();
    if (!features || !targets || !params) return set_error(KNN_EINVAL, "NULL pointer argument");
    if (n < 16 || epochs < 1 || batch < 1 || !(lr > 0.f)) return set_error(KNN_EINVAL, "bad training arguments");
    if (!(holdout > 0.f && holdout < 0.9f) || !(margin_quantile > 0.f && margin_quantile <= 1.f))
        return set_error(KNN_EINVAL, "holdout must be in (0, 0.9) and margin_quantile in (0, 1]");
    cudaStream_t st = opt ? static_cast<cudaStream_t>(opt->stream) : nullptr;
    // the last round(holdout n) rows are held out
    const int64_t n_hold = std::min<int64_t>(n - 1, std::llround(static_cast<double>(n) * holdout));
    const int64_t n_train = n - n_hold;
    Arena sz;
    sz.take<float>(N_TRAIN);
    sz.take<float>(N_TRAIN);
    sz.take<float>(N_TRAIN);
    sz.take<double>(1);
    sz.take<float>(n_hold);
    void* base = nullptr;
    KNN_TRY(workspace_get(sz.used(), &base));
    Arena ar(static_cast<char*>(base), sz.used());
    float* grad = ar.take<float>(N_TRAIN);
    float* m = ar.take<float>(N_TRAIN);
    float* v = ar.take<float>(N_TRAIN);
    double* loss = ar.take<double>(1);
    float* yh = ar.take<float>(n_hold);
    KNN_CK(cudaMemsetAsync(m, 0, N_TRAIN * sizeof(float), st));
    KNN_CK(cudaMemsetAsync(v, 0, N_TRAIN * sizeof(float), st));
    // standardisation from the training rows
    feature_stats_kernel<<<NF, 256, 0, st>>>(features, n_train, params);
    KNN_CK(cudaGetLastError());
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    int64_t step = 0;
    for (int e = 0; e < epochs; ++e) {
        double epoch_loss = 0.0;
        for (int64_t r0 = 0; r0 < n_train; r0 += batch) {
            const int64_t nb = std::min<int64_t>(batch, n_train - r0);
            KNN_CK(cudaMemsetAsync(grad, 0, N_TRAIN * sizeof(float), st));
            KNN_CK(cudaMemsetAsync(loss, 0, sizeof(double), st));
            mlp_kernel<true><<<static_cast<unsigned>((nb + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK), NH, 0, st>>>(
                features + r0 * NF, targets + r0, nb, nb, params, grad, loss, nullptr);
            ++step;
            const float c1 = 1.f - powf(b1, static_cast<float>(step));
            const float c2 = 1.f - powf(b2, static_cast<float>(step));
            adam_kernel<<<(N_TRAIN + 255) / 256, 256, 0, st>>>(params, grad, m, v, N_TRAIN, lr, b1, b2, eps, c1, c2);
            KNN_CK(cudaGetLastError());
            double l = 0.0;
            KNN_CK(cudaMemcpyAsync(&l, loss, sizeof(double), cudaMemcpyDeviceToHost, st));
            KNN_CK(cudaStreamSynchronize(st));
            epoch_loss += l * static_cast<double>(nb);
        }
        if (out_history) out_history[e] = static_cast<float>(epoch_loss / static_cast<double>(n_train));
    }
    // margin: the margin_quantile-th held-out residual t - y (at least 0)
    float margin = 0.f;
    if (n_hold > 0) {
        mlp_kernel<false><<<static_cast<unsigned>((n_hold + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK), NH, 0, st>>>(
            features + n_train * NF, nullptr, n_hold, n_hold, params, nullptr, nullptr, yh);
        KNN_CK(cudaGetLastError());
        std::vector<float> hy(static_cast<size_t>(n_hold)), ht(static_cast<size_t>(n_hold));
        KNN_CK(cudaMemcpyAsync(hy.data(), yh, n_hold * sizeof(float), cudaMemcpyDeviceToHost, st));
        KNN_CK(cudaMemcpyAsync(ht.data(), targets + n_train, n_hold * sizeof(float), cudaMemcpyDeviceToHost, st));
        KNN_CK(cudaStreamSynchronize(st));
        std::vector<float> res(static_cast<size_t>(n_hold));
        for (size_t i = 0; i < res.size(); ++i) res[i] = ht[i] - hy[i];
        std::sort(res.begin(), res.end());
        const size_t q = std::min(res.size() - 1, static_cast<size_t>(margin_quantile * (res.size() - 1) + 0.5));
        margin = std::max(0.f, res[q]);
    }
    KNN_CK(cudaMemcpyAsync(params + OFF_MARGIN, &margin, sizeof(float), cudaMemcpyHostToDevice, st));
    KNN_CK(cudaStreamSynchronize(st));
    return KNN_OK;
}

extern "C" int knn_mlp_predict(const float* features, int64_t n, const float* params, float* out_log_kth,
                               float* out_threshold, const knn_options* opt) {
    g_last_error.clear();
    if (!features || !params || (!out_log_kth && !out_threshold)) return set_error(KNN_EINVAL, "NULL pointer");
    if (n < 0) return set_error(KNN_EINVAL, "n must be >= 0");
    if (n == 0) return KNN_OK;
    cudaStream_t st = opt ? static_cast<cudaStream_t>(opt->stream) : nullptr;
    float* y = out_log_kth;
    if (!y) {
        Arena sz;
        sz.take<float>(n);
        void* base = nullptr;
        KNN_TRY(workspace_get(sz.used(), &base));
        Arena ar(static_cast<char*>(base), sz.used());
        y = ar.take<float>(n);
    }
    mlp_kernel<false><<<static_cast<unsigned>((n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK), NH, 0, st>>>(
        features, nullptr, n, n, params, nullptr, nullptr, y);
    KNN_CK(cudaGetLastError());
    if (out_threshold) {
        threshold_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(y, n, params, out_threshold);
        KNN_CK(cudaGetLastError());
    }
    KNN_CK(cudaStreamSynchronize(st));
    return KNN_OK;
}

// Parameter file: 8-byte magic "KNNMLP01", int32 features, int32 hidden, int32 count,
// then `count` little-endian FP32 parameters in the layout above.
namespace {
constexpr char MLP_MAGIC[8] = {'K', 'N', 'N', 'M', 'L', 'P', '0', '1'};
}

extern "C" int knn_mlp_save(const char* path, const float* params) {
    g_last_error.clear();
    if (!path || !params) return set_error(KNN_EINVAL, "NULL pointer argument");
    std::vector<float> h(N_PARAMS);
    if (is_device_pointer(params)) {
        KNN_CK(cudaMemcpy(h.data(), params, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(h.data(), params, N_PARAMS * sizeof(float));
    }
    FILE* f = std::fopen(path, "wb");
    if (!f) return set_error(KNN_EINVAL, "cannot open %s for writing", path);
    const int32_t hdr[3] = {NF, NH, N_PARAMS};
    bool ok = std::fwrite(MLP_MAGIC, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int32_t), 3, f) == 3 &&
              std::fwrite(h.data(), sizeof(float), N_PARAMS, f) == static_cast<size_t>(N_PARAMS);
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return set_error(KNN_EINVAL, "short write to %s", path);
    return KNN_OK;
}

extern "C" int knn_mlp_load(const char* path, float* params) {
    g_last_error.clear();
    if (!path || !params) return set_error(KNN_EINVAL, "NULL pointer argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return set_error(KNN_EINVAL, "cannot open %s", path);
    char magic[8] = {};
    int32_t hdr[3] = {};
    std::vector<float> h(N_PARAMS);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::fread(hdr, sizeof(int32_t), 3, f) == 3;
    ok = ok && std::memcmp(magic, MLP_MAGIC, 8) == 0 && hdr[0] == NF && hdr[1] == NH && hdr[2] == N_PARAMS;
    ok = ok && std::fread(h.data(), sizeof(float), N_PARAMS, f) == static_cast<size_t>(N_PARAMS);
    std::fclose(f);
    if (!ok) return set_error(KNN_EINVAL, "%s is not a parameter file of this network (%d-%d-1)", path, NF, NH);
    if (is_device_pointer(params)) {
        KNN_CK(cudaMemcpy(params, h.data(), N_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        std::memcpy(params, h.data(), N_PARAMS * sizeof(float));
    }
    return KNN_OK;
}
