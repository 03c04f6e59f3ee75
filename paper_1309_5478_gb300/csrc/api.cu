// C ABI entry points and the host-side runtime: argument checks, the per-device
// workspace, staging of host arrays, the slab loop of the plain form, and the
// exactness fallbacks.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "engine.h"
#include "internal.h"
#include "knn.h"
#include "tc_fused.h"

namespace knn {

thread_local std::string g_last_error;

int set_error(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

// ---------------------------------------------------------------------------
// workspace: one grow-only device buffer per device
// ---------------------------------------------------------------------------
namespace {
struct DevWs {
    void* ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_ws_mu;
std::unordered_map<int, DevWs> g_ws;
std::mutex g_stage_mu;
std::unordered_map<int, std::vector<DevWs>> g_stage;  // staging buffers of host arrays, per device and slot
thread_local int64_t g_ws_cap = 0;  // knn_options.max_workspace_bytes of the running call (0: none)
}  // namespace

WorkspaceCap::WorkspaceCap(int64_t bytes) : prev_(g_ws_cap) { g_ws_cap = bytes > 0 ? bytes : 0; }
WorkspaceCap::~WorkspaceCap() { g_ws_cap = prev_; }

int workspace_get(size_t bytes, void** out) {
    if (g_ws_cap > 0 && bytes > static_cast<size_t>(g_ws_cap))
        return set_error(KNN_ENOMEM, "the call needs %zu bytes of workspace, above max_workspace_bytes = %lld", bytes,
                         static_cast<long long>(g_ws_cap));
    int dev = 0;
    KNN_CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_ws_mu);
    DevWs& w = g_ws[dev];
    if (w.bytes < bytes) {
        if (w.ptr) {
            KNN_CK(cudaDeviceSynchronize());
            KNN_CK(cudaFree(w.ptr));
            w.ptr = nullptr;
            w.bytes = 0;
        }
        const size_t want = bytes + bytes / 8;
        cudaError_t e = cudaMalloc(&w.ptr, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            e = cudaMalloc(&w.ptr, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                w.ptr = nullptr;
                return set_error(KNN_ENOMEM, "workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
            }
            w.bytes = bytes;
        } else {
            w.bytes = want;
        }
    }
    *out = w.ptr;
    return KNN_OK;
}

void workspace_release_all() {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& kv : g_ws) {
        if (kv.second.ptr) {
            cudaSetDevice(kv.first);
            cudaDeviceSynchronize();
            cudaFree(kv.second.ptr);
        }
    }
    g_ws.clear();
    {
        std::lock_guard<std::mutex> lk2(g_stage_mu);
        for (auto& kv : g_stage) {
            cudaSetDevice(kv.first);
            cudaDeviceSynchronize();
            for (auto& w : kv.second)
                if (w.ptr) cudaFree(w.ptr);
        }
        g_stage.clear();
    }
    cudaSetDevice(cur);
    cudaGetLastError();
}

cudaError_t raise_smem_limit(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[{dev, kernel}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
    if (e == cudaSuccess) cur = bytes;
    return e;
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int pick_cap(int k, int km) {
    (void)k;
    const int extra = std::max(64, km / 2);
    int c = 32;
    while (c < km + extra) c <<= 1;
    return std::min(c, MAX_CAP);
}

namespace {

// Events and launch counts of one call (KNN_FLAG_TIMING).
struct Timing {
    bool on = false;
    std::vector<cudaEvent_t> gemm;  // pairs around each distance-kernel launch
    std::vector<cudaEvent_t> sel;   // pairs around each unfused select (plain form)
    std::vector<cudaEvent_t> rr;    // pairs around each re-rank launch of the plain form
    int64_t launches = 0;
    int32_t gemm_launches = 0;
    static int record(std::vector<cudaEvent_t>& v, bool on, cudaStream_t st) {
        if (!on) return KNN_OK;
        cudaEvent_t e;
        KNN_CK(cudaEventCreate(&e));
        v.push_back(e);
        KNN_CK(cudaEventRecord(e, st));
        return KNN_OK;
    }
    int record_gemm(cudaStream_t st, bool begin) {
        (void)begin;
        return record(gemm, on, st);
    }
    int record_sel(cudaStream_t st) { return record(sel, on, st); }
    int record_rr(cudaStream_t st) { return record(rr, on, st); }
    static float sum_ms(const std::vector<cudaEvent_t>& v) {
        float g = 0.f;
        for (size_t i = 0; i + 1 < v.size(); i += 2) {
            float t = 0.f;
            cudaEventElapsedTime(&t, v[i], v[i + 1]);
            g += t;
        }
        return g;
    }
    float gemm_ms() const { return sum_ms(gemm); }
    ~Timing() {
        for (auto& e : gemm) cudaEventDestroy(e);
        for (auto& e : sel) cudaEventDestroy(e);
        for (auto& e : rr) cudaEventDestroy(e);
    }
};

// ---------------------------------------------------------------------------
// plain form: FP32 SIMT GEMM slab -> unfused quick multi-select -> exact re-rank
// ---------------------------------------------------------------------------
struct PlainBuffers {
    float* D = nullptr;
    uint64_t* cand = nullptr;
    int32_t* count = nullptr;
    uint64_t* bound = nullptr;
    uint32_t* flags = nullptr;
    int64_t R = 0, ldn = 0;
    int km = 0, cap = 0;
};

void layout_plain_buffers(const Problem& pb, int64_t rows, Arena& ar, PlainBuffers& B) {
    B.km = static_cast<int>(std::min<int64_t>(pb.k + pb.m, pb.N - (pb.graph ? 1 : 0)));
    B.cap = pick_cap(pb.k, B.km);
    B.ldn = (pb.N + 31) / 32 * 32;
    const int64_t budget = pb.slab_bytes > 0 ? pb.slab_bytes : (int64_t(4) << 30);
    B.R = std::max<int64_t>(128, budget / (B.ldn * 4) / 128 * 128);
    B.R = std::min<int64_t>(B.R, (rows + 127) / 128 * 128);
    B.D = ar.take<float>(static_cast<size_t>(B.R) * B.ldn);
    B.cand = ar.take<uint64_t>(static_cast<size_t>(B.R) * B.cap);
    B.count = ar.take<int32_t>(B.R);
    B.bound = ar.take<uint64_t>(B.R);
    B.flags = ar.take<uint32_t>(B.R);
}

// Rows [0, M) of Q against the whole corpus. Row r excludes column self_col[r] (when
// self_col != nullptr) or r + self_offset (when self_offset >= 0).
int plain_pipeline(const Problem& pb, const float* Q, int64_t M, const int32_t* self_col, int64_t self_offset,
                   const float* cnorm2, const float* E, const float* thr, int32_t* out_idx, float* out_dist,
                   uint32_t* row_status, const PlainBuffers& B, RerankCounters* counters, cudaStream_t st,
                   Timing& tm) {
    for (int64_t r0 = 0; r0 < M; r0 += B.R) {
        const int64_t rows = std::min<int64_t>(B.R, M - r0);
        KNN_TRY(tm.record_gemm(st, true));
        KNN_CK(launch_gemm_simt(Q + r0 * pb.d, rows, 0, pb.C, pb.N, pb.d, cnorm2, nullptr, B.D, B.ldn, 0, st));
        KNN_TRY(tm.record_gemm(st, false));
        SelectParams sp{};
        sp.D = B.D;
        sp.ldd = B.ldn;
        sp.M = rows;
        sp.N = pb.N;
        sp.spec = select_spec(sp.N);
        sp.k = pb.k;
        sp.km = B.km;
        sp.cap = B.cap;
        sp.E = E + r0;
        sp.thr = thr ? thr + r0 : nullptr;
        sp.cand = B.cand;
        sp.count = B.count;
        sp.bound = B.bound;
        sp.flags = B.flags;
        sp.self_col = self_col ? self_col + r0 : nullptr;
        KNN_TRY(tm.record_sel(st));
        KNN_CK(launch_select_ex(sp, self_offset >= 0 ? self_offset + r0 : -1, false, st));
        KNN_TRY(tm.record_sel(st));
        RerankParams rp{};
        rp.Q = Q + r0 * pb.d;
        rp.C = pb.C;
        rp.M = rows;
        rp.N = pb.N;
        rp.d = pb.d;
        rp.k = pb.k;
        rp.km = sp.km;
        rp.cap = B.cap;
        rp.cand = B.cand;
        rp.count = B.count;
        rp.bound = B.bound;
        rp.flags = B.flags;
        rp.E = E + r0;
        rp.out_idx = out_idx + r0 * pb.k;
        rp.out_dist = out_dist + r0 * pb.k;
        rp.row_status = row_status + r0;
        rp.counters = counters;
        KNN_TRY(tm.record_rr(st));
        KNN_CK(launch_rerank(rp, st));
        KNN_TRY(tm.record_rr(st));
        tm.launches += 2 + rerank_launches(B.cap);
        tm.gemm_launches += 1;
    }
    return KNN_OK;
}

// Everything one call needs besides the form-specific buffers.
struct CommonLayout {
    PrepState ps{};
    float* E32 = nullptr;        // FP32-form bounds (the fallback's)
    uint32_t* row_status = nullptr;
    RerankCounters* counters = nullptr;
    int* status = nullptr;
    // fallback of uncertified rows
    int64_t fb_rows_max = 0, fp64_chunk = 0;
    int32_t* fb_rows = nullptr;
    float* fb_Q = nullptr;
    float* fb_E = nullptr;
    float* fb_T = nullptr;
    int32_t* fb_oi = nullptr;
    float* fb_od = nullptr;
    uint32_t* fb_status = nullptr;
    void* fb_xq = nullptr;       // gathered reduced-precision rows (second fused pass)
    float* fb_qscale = nullptr;  // and their FP8 scales
    PlainBuffers fb_plain{};
    double* fp64_scratch = nullptr;
    int64_t n_pad = 0;
    // integer inputs small enough that the error bounds can be zero: thresholds may then
    // be exact keys, whose float filter assumes columns in increasing order
    bool maybe_exact = false;
};

void layout_common(const Problem& pb, int prec, bool with_fallback_plain, Arena& ar, CommonLayout& L) {
    const bool same = pb.graph;
    PrepState& ps = L.ps;
    L.n_pad = (pb.N + 255) / 256 * 256;
    ps.gq = ar.take<PrepGlobals>(1);
    ps.gc = same ? ps.gq : ar.take<PrepGlobals>(1);
    ps.cnorm2 = ar.take<float>(L.n_pad);
    ps.qnorm2 = same ? ps.cnorm2 : ar.take<float>(pb.M);
    ps.E = ar.take<float>(pb.M);
    ps.thr_dprime = pb.thr ? ar.take<float>(pb.M) : nullptr;
    if (prec != P_FP32) {
        const int elem = prec == P_BF16 ? 2 : 1;
        const int per = 128 / elem;
        ps.d_pad = (pb.d + per - 1) / per * per;
        const size_t row_bytes = static_cast<size_t>(ps.d_pad) * elem;
        ps.cres = ar.take<float>(L.n_pad);
        ps.ctn = ar.take<float>(L.n_pad);
        ps.qres = same ? ps.cres : ar.take<float>(pb.M);
        ps.qtn = same ? ps.ctn : ar.take<float>(pb.M);
        ps.xc = ar.take<char>(row_bytes * pb.N);
        ps.xq = same ? ps.xc : ar.take<char>(row_bytes * pb.M);
        if (prec == P_FP8) {
            ps.cscale = ar.take<float>(L.n_pad);
            ps.qscale = same ? ps.cscale : ar.take<float>(pb.M);
        }
        L.E32 = ar.take<float>(pb.M);
    } else {
        ps.d_pad = pb.d;
        L.E32 = ps.E;
    }
    L.row_status = ar.take<uint32_t>(pb.M);
    L.counters = ar.take<RerankCounters>(1);
    L.status = ar.take<int>(1);
    L.fb_rows = ar.take<int32_t>(pb.M);
    // FP64 fallback scratch: rows of N doubles, up to 1 GiB (a quarter of a workspace cap)
    const int64_t fp64_budget = pb.slab_bytes > 0 ? pb.slab_bytes / 2 : (int64_t(1) << 30);
    L.fp64_chunk = std::max<int64_t>(1, std::min<int64_t>(pb.M, fp64_budget / (pb.N * 8)));
    L.fp64_scratch = ar.take<double>(static_cast<size_t>(L.fp64_chunk) * pb.N);
    if (with_fallback_plain) {
        L.fb_rows_max = std::min<int64_t>(pb.M, 16384);
        L.fb_Q = ar.take<float>(static_cast<size_t>(L.fb_rows_max) * pb.d);
        L.fb_E = ar.take<float>(L.fb_rows_max);
        L.fb_T = ar.take<float>(L.fb_rows_max);
        L.fb_oi = ar.take<int32_t>(static_cast<size_t>(L.fb_rows_max) * pb.k);
        L.fb_od = ar.take<float>(static_cast<size_t>(L.fb_rows_max) * pb.k);
        L.fb_status = ar.take<uint32_t>(L.fb_rows_max);
        if (prec != P_FP32) {
            L.fb_xq = ar.take<char>(static_cast<size_t>(L.fb_rows_max) * ps.d_pad * (prec == P_BF16 ? 2 : 1));
            if (prec == P_FP8) L.fb_qscale = ar.take<float>(L.fb_rows_max);
        }
        layout_plain_buffers(pb, L.fb_rows_max, ar, L.fb_plain);
    }
}

int prep_and_check(const Problem& pb, int prec, CommonLayout& L, cudaStream_t st, knn_stats* stats,
                   Timing& tm, bool sym_extra = false) {
    const PrepState& ps = L.ps;
    const bool same = pb.graph;
    KNN_CK(cudaMemsetAsync(ps.gq, 0, sizeof(PrepGlobals), st));
    if (!same) KNN_CK(cudaMemsetAsync(ps.gc, 0, sizeof(PrepGlobals), st));
    if (L.n_pad > pb.N) KNN_CK(cudaMemsetAsync(ps.cnorm2 + pb.N, 0xff, (L.n_pad - pb.N) * sizeof(float), st));
    const int ldq = prec == P_BF16 ? ps.d_pad : (prec == P_FP8 ? ps.d_pad : 0);
    KNN_CK(launch_prep(pb.C, pb.N, pb.d, prec, ps.cnorm2, ps.cres, ps.ctn, ps.xc, ldq, ps.cscale, ps.gc, st));
    ++tm.launches;
    if (!same) {
        KNN_CK(launch_prep(pb.Q, pb.M, pb.d, prec, ps.qnorm2, ps.qres, ps.qtn, ps.xq, ldq, ps.qscale, ps.gq, st));
        ++tm.launches;
    }
    KNN_CK(launch_bounds(ps.qnorm2, ps.qres, ps.qtn, pb.M, pb.d, ps.d_pad, prec, ps.gq, ps.gc, ps.E, st, sym_extra));
    ++tm.launches;
    if (prec != P_FP32) {
        KNN_CK(launch_bounds(ps.qnorm2, nullptr, nullptr, pb.M, pb.d, pb.d, P_FP32, ps.gq, ps.gc, L.E32, st));
        ++tm.launches;
    }
    if (pb.thr) {
        if (pb.thr_bound)
            KNN_CK(launch_bound_to_dprime(pb.thr, ps.qnorm2, ps.E, pb.M, pb.d, ps.thr_dprime, st));
        else
            KNN_CK(launch_threshold_to_dprime(pb.thr, ps.qnorm2, pb.M, ps.thr_dprime, st));
        ++tm.launches;
    }
    PrepGlobals hq{}, hc{};
    KNN_CK(cudaMemcpyAsync(&hq, ps.gq, sizeof(PrepGlobals), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaMemcpyAsync(&hc, ps.gc, sizeof(PrepGlobals), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaStreamSynchronize(st));
    if ((pb.flags & KNN_FLAG_CHECK_FINITE) && (hq.nonfinite || hc.nonfinite))
        return set_error(KNN_EINVAL, "input holds NaN or Inf (%u query rows, %u corpus rows)", hq.nonfinite,
                         hc.nonfinite);
    {
        float amax;
        uint32_t u = std::max(hq.max_abs, hc.max_abs);
        std::memcpy(&amax, &u, 4);
        L.maybe_exact = hq.noninteger == 0 && hc.noninteger == 0 && 4.0 * ps.d_pad * double(amax) * amax <= 16777216.0;
        if (stats) stats->exact_arithmetic = L.maybe_exact ? 1 : 0;
    }
    return KNN_OK;
}

// Host list of rows with `bit` set in status[0, M).
int rows_with(const uint32_t* status_d, int64_t M, uint32_t bit, cudaStream_t st, std::vector<int32_t>& rows) {
    std::vector<uint32_t> h(static_cast<size_t>(M));
    KNN_CK(cudaMemcpyAsync(h.data(), status_d, M * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaStreamSynchronize(st));
    rows.clear();
    for (int64_t i = 0; i < M; ++i)
        if (h[static_cast<size_t>(i)] & bit) rows.push_back(static_cast<int32_t>(i));
    return KNN_OK;
}

int exact_fp64_rows(const Problem& pb, const CommonLayout& L, const std::vector<int32_t>& rows, cudaStream_t st,
                    Timing& tm) {
    if (rows.empty()) return KNN_OK;
    if (pb.k > 2048) return set_error(KNN_EINTERNAL, "uncertified rows with k > 2048");
    KNN_CK(cudaMemcpyAsync(L.fb_rows, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    for (size_t r = 0; r < rows.size(); r += static_cast<size_t>(L.fp64_chunk)) {
        const int32_t n = static_cast<int32_t>(std::min<size_t>(L.fp64_chunk, rows.size() - r));
        KNN_CK(launch_exact_rows_fp64(pb.Q, pb.C, pb.N, pb.d, pb.k, pb.graph ? 1 : 0, L.fb_rows + r, n,
                                      L.fp64_scratch, pb.out_idx, pb.out_dist, st));
        ++tm.launches;
    }
    KNN_CK(cudaStreamSynchronize(st));
    return KNN_OK;
}

// Plain FP32 recompute of uncertified rows of a reduced-precision pass; rows the
// plain form cannot certify either go to FP64. Returns the number of FP64 rows.
int plain_fallback(const Problem& pb, const CommonLayout& L, const std::vector<int32_t>& rows, cudaStream_t st,
                   Timing& tm, int64_t* n_fp64) {
    std::vector<int32_t> still;
    for (size_t r0 = 0; r0 < rows.size(); r0 += static_cast<size_t>(L.fb_rows_max)) {
        const int32_t n = static_cast<int32_t>(std::min<size_t>(L.fb_rows_max, rows.size() - r0));
        KNN_CK(cudaMemcpyAsync(L.fb_rows, rows.data() + r0, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        KNN_CK(launch_gather_rows(pb.Q, pb.d, L.fb_rows, n, L.E32, nullptr, L.fb_Q, L.fb_E, nullptr, st));
        RerankCounters* ctr = L.counters;  // counts of the fallback are not reported separately
        KNN_TRY(plain_pipeline(pb, L.fb_Q, n, pb.graph ? L.fb_rows : nullptr, -1, L.ps.cnorm2, L.fb_E, nullptr,
                               L.fb_oi, L.fb_od, L.fb_status, L.fb_plain, ctr, st, tm));
        KNN_CK(launch_scatter_out(L.fb_rows, n, pb.k, L.fb_oi, L.fb_od, pb.out_idx, pb.out_dist, st));
        tm.launches += 2;
        std::vector<int32_t> bad;
        KNN_TRY(rows_with(L.fb_status, n, ROW_UNCERTIFIED, st, bad));
        for (int32_t b : bad) still.push_back(rows[r0 + static_cast<size_t>(b)]);
    }
    *n_fp64 = static_cast<int64_t>(still.size());
    return exact_fp64_rows(pb, L, still, st, tm);
}

void fill_stats(knn_stats* stats, const Problem& pb, const RerankCounters& hc, int64_t fallback, int prec, int fused,
                const Timing& tm, cudaEvent_t* ev) {
    if (!stats) return;
    stats->rows = pb.M;
    stats->candidates = static_cast<int64_t>(hc.candidates);
    stats->rows_truncated = static_cast<int64_t>(hc.truncated);
    stats->rows_uncertified = static_cast<int64_t>(hc.uncertified);
    stats->rows_fallback = fallback;
    stats->rows_fp64_ties = static_cast<int64_t>(hc.fp64_rows);
    stats->threshold_misses = static_cast<int64_t>(hc.threshold_miss);
    stats->candidates_inserted = static_cast<int64_t>(hc.inserted);
    {
        const uint32_t bits = static_cast<uint32_t>(hc.max_err_ratio);
        float r;
        std::memcpy(&r, &bits, sizeof(r));
        stats->max_error_ratio = r;
    }
    stats->rows_reranked_in_sweep = static_cast<int64_t>(hc.rows_in_sweep);
    stats->precision_used = prec;
    stats->fused_used = fused;
    stats->kernel_launches = tm.launches;
    stats->gemm_launches = tm.gemm_launches;
    stats->gemm_flops = 2.0 * double(pb.M) * double(pb.N) * double(pb.d);
    if (tm.on) {
        float a = 0, b = 0, c = 0, d = 0;
        cudaEventElapsedTime(&a, ev[0], ev[1]);
        cudaEventElapsedTime(&b, ev[1], ev[2]);
        cudaEventElapsedTime(&c, ev[2], ev[3]);
        cudaEventElapsedTime(&d, ev[3], ev[4]);
        stats->ms_prep = a;
        stats->ms_select = b;
        stats->ms_rerank = c;
        stats->ms_fallback = d;
        stats->ms_total = a + b + c + d;
        stats->ms_gemm = tm.gemm_ms();
    }
}

struct Events {
    cudaEvent_t ev[5] = {};
    bool on = false;
    int init(bool t) {
        on = t;
        if (on)
            for (auto& e : ev) KNN_CK(cudaEventCreate(&e));
        return KNN_OK;
    }
    int rec(int i, cudaStream_t st) {
        if (on) KNN_CK(cudaEventRecord(ev[i], st));
        return KNN_OK;
    }
    ~Events() {
        if (on)
            for (auto& e : ev) cudaEventDestroy(e);
    }
};

int run_plain(const Problem& pb, knn_stats* stats, cudaStream_t st) {
    CommonLayout L;
    PlainBuffers B;
    {
        Arena sz;
        layout_common(pb, P_FP32, false, sz, L);
        layout_plain_buffers(pb, pb.M, sz, B);
        void* base = nullptr;
        KNN_TRY(workspace_get(sz.used(), &base));
        Arena ar(static_cast<char*>(base), sz.used());
        L = CommonLayout{};
        B = PlainBuffers{};
        layout_common(pb, P_FP32, false, ar, L);
        layout_plain_buffers(pb, pb.M, ar, B);
    }
    Timing tm;
    tm.on = stats && (pb.flags & KNN_FLAG_TIMING);
    Events ev;
    KNN_TRY(ev.init(tm.on));
    KNN_TRY(ev.rec(0, st));
    KNN_TRY(prep_and_check(pb, P_FP32, L, st, stats, tm));
    KNN_CK(cudaMemsetAsync(L.counters, 0, sizeof(RerankCounters), st));
    KNN_TRY(ev.rec(1, st));
    // a bounding threshold only saves work in the fused sweep; the plain form runs without it
    KNN_TRY(plain_pipeline(pb, pb.Q, pb.M, nullptr, pb.graph ? 0 : -1, L.ps.cnorm2, L.ps.E,
                           pb.thr_bound ? nullptr : L.ps.thr_dprime, pb.out_idx, pb.out_dist, L.row_status, B,
                           L.counters, st, tm));
    KNN_TRY(ev.rec(2, st));
    KNN_TRY(ev.rec(3, st));
    RerankCounters hc{};
    KNN_CK(cudaMemcpyAsync(&hc, L.counters, sizeof(hc), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaStreamSynchronize(st));
    int64_t fallback = 0;
    if (hc.uncertified > 0 && !(pb.flags & KNN_FLAG_NO_FALLBACK)) {
        std::vector<int32_t> rows;
        KNN_TRY(rows_with(L.row_status, pb.M, ROW_UNCERTIFIED, st, rows));
        KNN_TRY(exact_fp64_rows(pb, L, rows, st, tm));
        fallback = static_cast<int64_t>(rows.size());
    }
    KNN_TRY(ev.rec(4, st));
    KNN_CK(cudaStreamSynchronize(st));
    fill_stats(stats, pb, hc, fallback, KNN_FP32, 0, tm, ev.ev);
    if (stats) {
        stats->list_capacity = B.cap;
        if (tm.on) {
            // the slabs interleave GEMM, select and re-rank: report each kernel's own device time
            stats->ms_select = Timing::sum_ms(tm.sel);
            stats->ms_rerank = Timing::sum_ms(tm.rr);
        }
    }
    return KNN_OK;
}

// Sampled rows of the band probe and the smallest problem it runs on (M N pairs).
constexpr int PROBE_ROWS = 64;
constexpr double PROBE_MIN_PAIRS = 1073741824.0;  // 2^30

struct ProbeBuffers {
    int32_t* rows = nullptr;   // PROBE_ROWS sampled query rows
    float* Qs = nullptr;       // their coordinates
    float* Es = nullptr;       // their reduced-precision bounds
    float* D = nullptr;        // PROBE_ROWS x N FP32 d'
    int32_t* oi = nullptr;     // PROBE_ROWS x km
    float* ov = nullptr;
    uint32_t* fl = nullptr;
    int32_t* cnt = nullptr;    // 2 x PROBE_ROWS: band counts with 2E, then with 4E
    float* edge = nullptr;     // band edges of the sampled rows as squared distances
};

// List capacity of the fused form from the band of a few sampled rows: the 90th
// percentile band plus a quarter, plus room for one half-tile of insertions from both
// warps of a row (128) and slack (32), but never below the default for k + m.
// With spec_d2 (speculative thresholds on) it also proposes a start threshold for every
// row: the largest sampled band edge (a squared distance) plus twice its distance from
// the median edge. For points whose bands are alike this starts every row's sweep near
// its final threshold; a row whose band lies beyond it is caught at the end of the
// sweep (truncated, re-rank certificate, second pass). Where the edges spread widely
// the proposal is loose and costs nothing.
int probe_cap(const Problem& pb, int prec, int km, const CommonLayout& L, const ProbeBuffers& pr, cudaStream_t st,
              Timing& tm, int* cap_out, float* spec_d2, int* keys_le_t = nullptr) {
    std::vector<int32_t> rows(PROBE_ROWS);
    for (int i = 0; i < PROBE_ROWS; ++i) rows[i] = static_cast<int32_t>((pb.M * (2 * i + 1)) / (2 * PROBE_ROWS));
    KNN_CK(cudaMemcpyAsync(pr.rows, rows.data(), PROBE_ROWS * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    KNN_CK(launch_gather_rows(pb.Q, pb.d, pr.rows, PROBE_ROWS, L.ps.E, nullptr, pr.Qs, pr.Es, nullptr, st));
    KNN_CK(launch_gemm_simt(pr.Qs, PROBE_ROWS, 0, pb.C, pb.N, pb.d, L.ps.cnorm2, nullptr, pr.D, pb.N, 0, st));
    SelectParams sp{};
    sp.D = pr.D;
    sp.ldd = pb.N;
    sp.M = PROBE_ROWS;
    sp.N = pb.N;
    sp.spec = select_spec(sp.N);
    sp.k = km;
    sp.km = km;
    sp.cap = km;
    sp.flags = pr.fl;
    sp.self_col = pb.graph ? pr.rows : nullptr;
    KNN_CK(launch_select_topk(sp, pr.oi, pr.ov, st));
    KNN_CK(launch_band_count(pr.D, PROBE_ROWS, pb.N, pb.N, pr.ov, pb.k, km, pr.Es, sp.self_col, L.ps.qnorm2,
                             pr.rows, pr.cnt, pr.cnt + PROBE_ROWS, pr.edge, st));
    tm.launches += 4;
    std::vector<int32_t> cnt(PROBE_ROWS), cnt4(PROBE_ROWS);
    std::vector<float> edge(PROBE_ROWS);
    KNN_CK(cudaMemcpyAsync(cnt.data(), pr.cnt, PROBE_ROWS * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaMemcpyAsync(cnt4.data(), pr.cnt + PROBE_ROWS, PROBE_ROWS * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaMemcpyAsync(edge.data(), pr.edge, PROBE_ROWS * sizeof(float), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaStreamSynchronize(st));
    if (spec_d2) {
        std::sort(edge.begin(), edge.end());
        const float med = edge[PROBE_ROWS / 2], mx = edge[PROBE_ROWS - 1];
        const float t = mx + 2.f * (mx - med) + 1e-6f * std::fabs(mx);
        *spec_d2 = std::isfinite(t) ? t : __builtin_huge_valf();
        if (keys_le_t && std::isfinite(t)) {
            // the most keys any sampled row has at or below t (its inbox in the symmetric form)
            KNN_CK(launch_count_le(pr.D, PROBE_ROWS, pb.N, pb.N, t, L.ps.qnorm2, pr.rows,
                                   pb.graph ? pr.rows : nullptr, pr.cnt, st));
            ++tm.launches;
            std::vector<int32_t> le(PROBE_ROWS);
            KNN_CK(cudaMemcpyAsync(le.data(), pr.cnt, PROBE_ROWS * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            KNN_CK(cudaStreamSynchronize(st));
            *keys_le_t = *std::max_element(le.begin(), le.end());
        }
    }
    std::sort(cnt.begin(), cnt.end());
    std::sort(cnt4.begin(), cnt4.end());
    const int band = cnt[(PROBE_ROWS * 9) / 10];
    const int band4 = cnt4[(PROBE_ROWS * 9) / 10];
    const int base = std::min(std::max((band + band / 4 + 160 + 31) / 32 * 32, fused_cap(pb.k, km)), FUSED_CAP_WIDE);
    // a truncating shrink in the sweep keeps cap / 2 keys: keep that above the band the lists
    // can reach on approximate values (exact v_k + 4E), or rows with dense neighbourhoods are
    // truncated inside their band and end uncertified -- but never at the price of a stage of
    // the GEMM's operand pipeline (the lists share its shared memory)
    int cap = std::min(std::max(base, (2 * band4 + 31) / 32 * 32), FUSED_CAP_WIDE);
    // nor at the price of the re-rank warps' buffers, where they fit at the base capacity
    const bool rr = fused_stages(base, prec, true) == fused_stages(base, prec, false);
    const int stages = fused_stages(base, prec, rr);
    while (cap > base && fused_stages(cap, prec, rr) < stages) cap -= 32;
    *cap_out = cap;
    return KNN_OK;
}

// Second fused pass over the rows the first could not certify (a band wider than the
// list, or a threshold that cut into the answer): the widest lists and no threshold,
// over the gathered rows, in chunks that fit the first pass's candidate buffer. Rows it
// cannot certify either are returned in `still`.
// List capacity of the second fused pass after a first pass with capacity cap.
int retry_cap(int cap) { return std::min(FUSED_CAP_MAX, std::max(FUSED_CAP_WIDE, cap + 256)); }

int fused_retry(const Problem& pb, int prec, const CommonLayout& L, const FusedParams& first, size_t cand_keys,
                const std::vector<int32_t>& rows, int sms, cudaStream_t st, Timing& tm, std::vector<int32_t>& still) {
    const int cap2 = retry_cap(first.cap);
    const int stages2 = fused_stages(cap2, prec);
    const int64_t chunk = std::min<int64_t>(L.fb_rows_max, static_cast<int64_t>(cand_keys / cap2));
    if (stages2 == 0 || chunk < 1) {
        still = rows;
        return KNN_OK;
    }
    const int row_bytes = L.ps.d_pad * (prec == P_BF16 ? 2 : 1);
    for (size_t r0 = 0; r0 < rows.size(); r0 += static_cast<size_t>(chunk)) {
        const int32_t n = static_cast<int32_t>(std::min<size_t>(chunk, rows.size() - r0));
        KNN_CK(cudaMemcpyAsync(L.fb_rows, rows.data() + r0, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        KNN_CK(launch_gather_rows(pb.Q, pb.d, L.fb_rows, n, L.ps.E, nullptr, L.fb_Q, L.fb_E, nullptr, st));
        KNN_CK(launch_gather_qrows(L.ps.xq, row_bytes, prec == P_FP8 ? L.ps.qscale : nullptr, L.fb_rows, n, L.fb_xq,
                                   L.fb_qscale, st));
        FusedParams fp = first;
        fp.rr_on = 0;  // the second pass re-ranks its gathered rows after the kernel
        fp.sym = 0;    // and sweeps every column of its rows
        fp.inbox = nullptr;
        fp.inbox_cnt = nullptr;
        fp.xq = L.fb_xq;
        fp.M = n;
        fp.cap = cap2;
        fp.cap_max = cap2;
        fp.stages = stages2;
        fp.E = L.fb_E;
        fp.thr = nullptr;
        fp.q_inv_scale = L.fb_qscale;
        fp.self_offset = -1;
        fp.self_col = pb.graph ? L.fb_rows : nullptr;
        fp.spec = 0;
        fp.perm_a = 1;
        fp.qnorm2 = nullptr;
        fp.spec_d2 = __builtin_huge_valf();
        fp.n_items = static_cast<int32_t>((n + 127) / 128);
        KNN_CK(launch_fused(fp, prec, std::min(sms, fp.n_items), st));
        int hstatus = 0;
        KNN_CK(cudaMemcpyAsync(&hstatus, L.status, sizeof(int), cudaMemcpyDeviceToHost, st));
        KNN_CK(cudaStreamSynchronize(st));
        if (hstatus != 0) return set_error(KNN_ETIMEOUT, "the fused kernel stopped: a device-side wait timed out");
        RerankParams rp{};
        rp.Q = L.fb_Q;
        rp.C = pb.C;
        rp.M = n;
        rp.N = pb.N;
        rp.d = pb.d;
        rp.k = pb.k;
        rp.km = first.km;
        rp.cap = cap2;
        rp.cand = first.cand;
        rp.count = first.count;
        rp.bound = first.bound;
        rp.flags = first.flags;
        rp.E = L.fb_E;
        rp.out_idx = L.fb_oi;
        rp.out_dist = L.fb_od;
        rp.row_status = L.fb_status;
        rp.counters = L.counters;  // the first pass's counts were read before
        KNN_CK(launch_rerank(rp, st));
        KNN_CK(launch_scatter_out(L.fb_rows, n, pb.k, L.fb_oi, L.fb_od, pb.out_idx, pb.out_dist, st));
        tm.launches += 4 + rerank_launches(cap2);
        std::vector<int32_t> bad;
        KNN_TRY(rows_with(L.fb_status, n, ROW_UNCERTIFIED, st, bad));
        for (int32_t b : bad) still.push_back(rows[r0 + static_cast<size_t>(b)]);
    }
    return KNN_OK;
}

// Speculative thresholds pay off when a row block's sweep is long; below this many
// corpus points the plain running threshold is kept. KNN_SPECULATE=0 turns them off.
constexpr int64_t SPEC_MIN_N = 16384;

bool speculate(const Problem& pb) {
    if (pb.spec >= 0) return pb.spec != 0 && pb.N >= 2 * 256;
    if (const char* e = std::getenv("KNN_SPECULATE")) return std::atoi(e) != 0 && pb.N >= 2 * 256;
    return pb.N >= SPEC_MIN_N;
}

// The probe's start threshold (part of speculation); KNN_SPEC_START=0 turns it off alone.
bool spec_start() {
    const char* e = std::getenv("KNN_SPEC_START");
    return !e || std::atoi(e) != 0;
}

// Tile stride of the sweep order ct * a mod n: a odd, coprime to n, near 0.618 n, so that
// any prefix of the sweep is spread over the whole corpus (speculation assumes the
// columns seen first are a fair sample of the row's distances).
int tile_stride(int64_t n) {
    if (n <= 2) return 1;
    auto gcd = [](int64_t a, int64_t b) {
        while (b) {
            const int64_t t = a % b;
            a = b;
            b = t;
        }
        return a;
    };
    for (int64_t a = static_cast<int64_t>(0.6180339887 * static_cast<double>(n)) | 1; a > 1; a -= 2)
        if (gcd(a, n) == 1) return static_cast<int>(a);
    return 1;
}

// The symmetric form of a k-NN graph (half the distance product; KNN_SYMMETRIC=0 turns it
// off, 2 takes it even where the probe expects inboxes to overflow): it needs the probe's
// start threshold, which it also takes as the threshold of the transposed pairs.
int symmetric_mode() {
    const char* e = std::getenv("KNN_SYMMETRIC");
    return e ? std::atoi(e) : 1;
}
bool symmetric_enabled() { return symmetric_mode() != 0; }

// Pairs (i, j) the symmetric form's fused launch computes: row block rb (128 rows) sweeps
// the columns from 256 (rb / 2) on.
double symmetric_pairs(int64_t M, int64_t N) {
    double pairs = 0.0;
    for (int64_t rb = 0; rb * 128 < M; ++rb) {
        const int64_t rows = std::min<int64_t>(128, M - rb * 128);
        pairs += static_cast<double>(rows) * static_cast<double>(N - 256 * (rb / 2));
    }
    return pairs;
}

// Polls of a bounded device-side wait before a kernel gives up (0: the kernel's default).
// KNN_WAIT_LIMIT overrides it, so that the give-up path can be exercised.
long long wait_limit() {
    const char* e = std::getenv("KNN_WAIT_LIMIT");
    return e ? std::max(1ll, std::atoll(e)) : 0ll;
}

// Whether the fused kernel's re-rank warps take the rows of finished row blocks during the
// sweep: they need 16-byte aligned rows with d % 4 == 0, at least two row blocks per CTA
// (the last one is always left to the re-rank launch), and shared memory that costs the
// GEMM no pipeline stage. KNN_RERANK_IN_SWEEP=0 turns it off.
bool rerank_in_sweep(const Problem& pb, int prec, int cap, int64_t nrb, int grid) {
    if (const char* e = std::getenv("KNN_RERANK_IN_SWEEP"))
        if (std::atoi(e) == 0) return false;
    const bool vec = pb.d % 4 == 0 && reinterpret_cast<uintptr_t>(pb.Q) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(pb.C) % 16 == 0;
    return vec && nrb >= 2 * static_cast<int64_t>(grid) && fused_stages(cap, prec, true) == fused_stages(cap, prec, false);
}

int run_fused(const Problem& pb, int prec, knn_stats* stats, cudaStream_t st) {
    CommonLayout L;
    uint64_t* cand = nullptr;
    int32_t* count = nullptr;
    uint64_t* bound = nullptr;
    uint32_t* flags = nullptr;
    const int km = static_cast<int>(std::min<int64_t>(pb.k + pb.m, pb.N - (pb.graph ? 1 : 0)));
    int cap = fused_cap(pb.k, km);
    // a large problem first measures its band on sampled rows and may take a larger list; a
    // search within a bounding threshold (a streamed chunk after the first) starts at the bound
    // instead, and few of its points lie within it
    const bool probe = static_cast<double>(pb.M) * static_cast<double>(pb.N) >= PROBE_MIN_PAIRS &&
                       pb.M >= 4 * PROBE_ROWS && fused_stages(FUSED_CAP_WIDE, prec) > 0 && !pb.thr_bound;
    // tuning override: a list capacity between the default for k + m and the maximum
    int cap_env = 0;
    if (const char* e = std::getenv("KNN_FUSED_CAP"))
        cap_env = std::min(FUSED_CAP_MAX, std::max(cap, (std::atoi(e) + 31) / 32 * 32));
    const int cap_alloc = probe ? std::max(FUSED_CAP_WIDE, cap) : std::max(cap, cap_env);
    int dev = 0, sms = 0;
    KNN_CK(cudaGetDevice(&dev));
    KNN_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t nrb = (pb.M + 127) / 128;
    const int grid = static_cast<int>(std::min<int64_t>(sms, nrb));
    uint64_t* scratch = nullptr;
    ProbeBuffers pr;
    // symmetric graph form: transposed pairs land in per-row inboxes
    const bool sym_want = pb.graph && probe && speculate(pb) && spec_start() && symmetric_enabled();
    const int cap_in = FUSED_CAP_WIDE;
    uint64_t* inbox = nullptr;
    int32_t* inbox_cnt = nullptr;
    auto layout = [&](Arena& ar) {
        layout_common(pb, prec, true, ar, L);
        cand = ar.take<uint64_t>(static_cast<size_t>(pb.M) * cap_alloc);
        count = ar.take<int32_t>(pb.M);
        bound = ar.take<uint64_t>(pb.M);
        flags = ar.take<uint32_t>(pb.M);
        scratch = ar.take<uint64_t>(fused_scratch_words(FUSED_CAP_MAX, grid));  // also serves the second pass
        if (sym_want) {
            inbox = ar.take<uint64_t>(static_cast<size_t>(pb.M) * cap_in);
            inbox_cnt = ar.take<int32_t>(pb.M);
        }
        if (probe) {
            pr.rows = ar.take<int32_t>(PROBE_ROWS);
            pr.Qs = ar.take<float>(static_cast<size_t>(PROBE_ROWS) * pb.d);
            pr.Es = ar.take<float>(PROBE_ROWS);
            pr.D = ar.take<float>(static_cast<size_t>(PROBE_ROWS) * pb.N);
            pr.oi = ar.take<int32_t>(static_cast<size_t>(PROBE_ROWS) * km);
            pr.ov = ar.take<float>(static_cast<size_t>(PROBE_ROWS) * km);
            pr.fl = ar.take<uint32_t>(PROBE_ROWS);
            pr.cnt = ar.take<int32_t>(2 * PROBE_ROWS);
            pr.edge = ar.take<float>(PROBE_ROWS);
        }
    };
    {
        Arena sz;
        layout(sz);
        void* base = nullptr;
        KNN_TRY(workspace_get(sz.used(), &base));
        Arena ar(static_cast<char*>(base), sz.used());
        L = CommonLayout{};
        layout(ar);
    }
    Timing tm;
    tm.on = stats && (pb.flags & KNN_FLAG_TIMING);
    Events ev;
    KNN_TRY(ev.init(tm.on));
    KNN_TRY(ev.rec(0, st));
    KNN_TRY(prep_and_check(pb, prec, L, st, stats, tm, sym_want));
    KNN_CK(cudaMemsetAsync(L.counters, 0, sizeof(RerankCounters), st));
    KNN_CK(cudaMemsetAsync(L.status, 0, sizeof(int), st));
    float spec_d2 = __builtin_huge_valf();
    const bool spec = speculate(pb);
    int keys_le_t = 0;
    if (probe)
        KNN_TRY(probe_cap(pb, prec, km, L, pr, st, tm, &cap, spec && spec_start() ? &spec_d2 : nullptr,
                          sym_want ? &keys_le_t : nullptr));
    if (cap_env > 0) cap = cap_env;
    const int stages = fused_stages(cap, prec);
    if (stages == 0) return set_error(KNN_EINTERNAL, "fused list capacity %d does not fit", cap);
    KNN_TRY(ev.rec(1, st));

    FusedParams fp{};
    fp.xq = L.ps.xq;
    fp.xc = L.ps.xc;
    fp.M = pb.M;
    fp.N = pb.N;
    fp.k_bytes = L.ps.d_pad * (prec == P_BF16 ? 2 : 1);
    fp.k = pb.k;
    fp.km = km;
    fp.cap = cap;
    fp.cnorm2 = L.ps.cnorm2;
    fp.E = L.ps.E;
    fp.thr = L.ps.thr_dprime;
    fp.thr_bound = pb.thr_bound ? 1 : 0;
    fp.q_inv_scale = L.ps.qscale;
    fp.c_inv_scale = L.ps.cscale;
    fp.self_offset = pb.graph ? 0 : -1;
    fp.cand = cand;
    fp.count = count;
    fp.bound = bound;
    fp.flags = flags;
    fp.status = L.status;
    fp.scratch = scratch;
    fp.inserted = &L.counters->inserted;
    fp.stages = stages;
    fp.cap_max = cap;
    fp.n_items = static_cast<int32_t>(nrb);
    fp.spec = spec ? 1 : 0;
    fp.perm_a = fp.spec && !L.maybe_exact ? tile_stride((pb.N + 255) / 256) : 1;
    fp.qnorm2 = L.ps.qnorm2;
    fp.spec_d2 = spec_d2;
    fp.wait_limit = wait_limit();
    // the symmetric form needs the inboxes to hold a row's transposed pairs: where sampled rows
    // already have more keys below the threshold than three quarters of an inbox (crowded or
    // unevenly dense data), the full sweep is kept
    const bool sym = sym_want && std::isfinite(spec_d2) && (keys_le_t <= (3 * cap_in) / 4 || symmetric_mode() == 2);
    if (sym) {
        // no speculative ranks mid-sweep: the start threshold alone is speculative, and the
        // certificate checks it for every row (rows it rejects take the second pass)
        fp.sym = 1;
        fp.sym_t = spec_d2;
        fp.inbox = inbox;
        fp.inbox_cnt = inbox_cnt;
        fp.cap_in = cap_in;
        fp.c2max_bits = &L.ps.gc->max_norm2;
        fp.spec = 0;
        fp.perm_a = 1;
        KNN_CK(cudaMemsetAsync(inbox_cnt, 0, static_cast<size_t>(pb.M) * sizeof(int32_t), st));
    }

    RerankParams rp{};
    rp.Q = pb.Q;
    rp.C = pb.C;
    rp.M = pb.M;
    rp.N = pb.N;
    rp.d = pb.d;
    rp.k = pb.k;
    rp.km = km;
    rp.cap = cap;
    rp.cand = cand;
    rp.count = count;
    rp.bound = bound;
    rp.flags = flags;
    rp.E = L.ps.E;
    rp.out_idx = pb.out_idx;
    rp.out_dist = pb.out_dist;
    rp.row_status = L.row_status;
    rp.counters = L.counters;
    rp.status = L.status;  // nothing is re-ranked after the fused kernel gave up
    if (sym) {
        rp.inbox = inbox;
        rp.inbox_cnt = inbox_cnt;
        rp.cap_in = cap_in;
    }
    // the re-rank of finished row blocks overlaps the sweep of later ones; the launch after
    // the kernel takes the rows the sweep's re-rank warps did not (a row of the symmetric form
    // is complete only when every row block above it has passed its columns)
    fp.rr_on = !sym && rerank_in_sweep(pb, prec, cap, nrb, grid) ? 1 : 0;
    fp.rr = rp;
    rp.skip_done = fp.rr_on;
    if (fp.rr_on) KNN_CK(cudaMemsetAsync(L.row_status, 0, static_cast<size_t>(pb.M) * sizeof(uint32_t), st));
    KNN_TRY(tm.record_gemm(st, true));
    KNN_CK(launch_fused(fp, prec, grid, st));
    KNN_TRY(tm.record_gemm(st, false));
    ++tm.launches;
    ++tm.gemm_launches;
    KNN_TRY(ev.rec(2, st));
    KNN_CK(launch_rerank(rp, st));
    tm.launches += rerank_launches(cap + (sym ? cap_in : 0));
    KNN_TRY(ev.rec(3, st));
    int hstatus = 0;
    RerankCounters hc{};
    KNN_CK(cudaMemcpyAsync(&hstatus, L.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaMemcpyAsync(&hc, L.counters, sizeof(hc), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaStreamSynchronize(st));
    if (hstatus != 0) return set_error(KNN_ETIMEOUT, "the fused kernel stopped: a device-side wait timed out");
    int64_t fallback = 0;
    if (hc.uncertified > 0 && !(pb.flags & KNN_FLAG_NO_FALLBACK)) {
        std::vector<int32_t> rows;
        KNN_TRY(rows_with(L.row_status, pb.M, ROW_UNCERTIFIED, st, rows));
        std::vector<int32_t> still;
        if (retry_cap(cap) > cap || pb.thr || fp.spec)
            KNN_TRY(fused_retry(pb, prec, L, fp, static_cast<size_t>(pb.M) * cap_alloc, rows, sms, st, tm, still));
        else
            still = rows;
        int64_t n64 = 0;
        KNN_TRY(plain_fallback(pb, L, still, st, tm, &n64));
        fallback = static_cast<int64_t>(rows.size());
    }
    KNN_TRY(ev.rec(4, st));
    KNN_CK(cudaStreamSynchronize(st));
    // the fallback's re-rank adds to the counters after they were read: report the first pass
    fill_stats(stats, pb, hc, fallback, prec == P_BF16 ? KNN_BF16 : KNN_FP8_E4M3, 1, tm, ev.ev);
    if (stats) {
        stats->list_capacity = cap;
        stats->symmetric = sym ? 1 : 0;
        if (sym) stats->gemm_flops = 2.0 * symmetric_pairs(pb.M, pb.N) * pb.d;
    }
    return KNN_OK;
}

// ---------------------------------------------------------------------------
// host-array staging
// ---------------------------------------------------------------------------
// Device copies of host arrays. The buffers are cached per device and slot (the i-th array a
// call stages) and only grow, like the workspace, so repeated calls on host arrays neither
// allocate nor free (cudaFree would also synchronise the device); knn_shutdown releases them.
struct Staged {
    int slot = 0;
    cudaStream_t stream = nullptr;
    bool finished = false;
    // a call that returns early may leave copies into the cached buffers in flight: they end
    // before the buffers can serve another call
    ~Staged() {
        if (slot > 0 && !finished) cudaStreamSynchronize(stream);
    }
    int take(size_t bytes, void** d) {
        int dev = 0;
        KNN_CK(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lk(g_stage_mu);
        std::vector<DevWs>& v = g_stage[dev];
        if (static_cast<int>(v.size()) <= slot) v.resize(static_cast<size_t>(slot) + 1);
        DevWs& w = v[static_cast<size_t>(slot++)];
        if (w.bytes < bytes) {
            if (w.ptr) {
                KNN_CK(cudaDeviceSynchronize());
                KNN_CK(cudaFree(w.ptr));
                w.ptr = nullptr;
                w.bytes = 0;
            }
            cudaError_t e = cudaMalloc(&w.ptr, bytes ? bytes : 1);
            if (e != cudaSuccess) {
                cudaGetLastError();
                w.ptr = nullptr;
                return set_error(KNN_ENOMEM, "staging %zu bytes: %s", bytes, cudaGetErrorString(e));
            }
            w.bytes = bytes ? bytes : 1;
        }
        *d = w.ptr;
        return KNN_OK;
    }
    int in(const void* p, size_t bytes, cudaStream_t st, const void** out) {
        if (!p || is_device_pointer(p)) {
            *out = p;
            return KNN_OK;
        }
        void* d = nullptr;
        stream = st;
        KNN_TRY(take(bytes, &d));
        KNN_CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, st));
        *out = d;
        return KNN_OK;
    }
    // Output: returns a device buffer; copy_back() moves it to the host pointer.
    std::vector<std::tuple<void*, void*, size_t>> outs;
    int out(void* p, size_t bytes, void** dev) {
        if (is_device_pointer(p)) {
            *dev = p;
            return KNN_OK;
        }
        void* d = nullptr;
        KNN_TRY(take(bytes, &d));
        outs.emplace_back(p, d, bytes);
        *dev = d;
        return KNN_OK;
    }
    int copy_back(cudaStream_t st) {
        stream = st;
        for (auto& t : outs)
            KNN_CK(cudaMemcpyAsync(std::get<0>(t), std::get<1>(t), std::get<2>(t), cudaMemcpyDeviceToHost, st));
        KNN_CK(cudaStreamSynchronize(st));
        finished = true;
        return KNN_OK;
    }
};

cudaStream_t stream_of(const knn_options* o) { return o ? static_cast<cudaStream_t>(o->stream) : nullptr; }

knn_options defaults() {
    knn_options o;
    knn_options_init(&o);
    return o;
}

int validate_args(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k, const int32_t* out_idx,
                  const float* out_dist, const knn_options& opt, bool graph) {
    if (!C || !out_idx || !out_dist || (!graph && !Q)) return set_error(KNN_EINVAL, "NULL pointer argument");
    if (d < 1) return set_error(KNN_EINVAL, "d must be >= 1 (got %d)", d);
    if (k < 1) return set_error(KNN_EINVAL, "k must be >= 1 (got %d)", k);
    if (N < 1 || N >= (int64_t(1) << 31)) return set_error(KNN_EINVAL, "N must be in [1, 2^31) (got %lld)", (long long)N);
    if (M < 0) return set_error(KNN_EINVAL, "M must be >= 0");
    if (graph && M != N) return set_error(KNN_EINVAL, "a k-NN graph needs M == N");
    if (graph && k > N - 1) return set_error(KNN_EINVAL, "k must be <= N - 1 for a k-NN graph (k=%d, N=%lld)", k, (long long)N);
    if (!graph && k > N) return set_error(KNN_EINVAL, "k must be <= N (k=%d, N=%lld)", k, (long long)N);
    if (k > MAX_K) return set_error(KNN_EINVAL, "k above %d is not supported (got %d)", MAX_K, k);
    if (opt.rerank_extra < 0) return set_error(KNN_EINVAL, "rerank_extra must be >= 0");
    return KNN_OK;
}

int search_impl(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k, int32_t* out_idx,
                float* out_dist, const knn_options* opt_in, bool graph) {
    g_last_error.clear();
    const knn_options opt = opt_in ? *opt_in : defaults();
    KNN_TRY(validate_args(Q, M, C, N, d, k, out_idx, out_dist, opt, graph));
    if (M == 0) return KNN_OK;
    const WorkspaceCap cap_guard(opt.max_workspace_bytes);
    cudaStream_t st = stream_of(&opt);
    Staged sg;
    const void *Qd = nullptr, *Cd = nullptr, *Td = nullptr;
    KNN_TRY(sg.in(C, static_cast<size_t>(N) * d * sizeof(float), st, &Cd));
    if (graph) {
        Qd = Cd;
    } else {
        KNN_TRY(sg.in(Q, static_cast<size_t>(M) * d * sizeof(float), st, &Qd));
    }
    if (opt.row_threshold) KNN_TRY(sg.in(opt.row_threshold, static_cast<size_t>(M) * sizeof(float), st, &Td));
    void *oi = nullptr, *od = nullptr;
    KNN_TRY(sg.out(out_idx, static_cast<size_t>(M) * k * sizeof(int32_t), &oi));
    KNN_TRY(sg.out(out_dist, static_cast<size_t>(M) * k * sizeof(float), &od));
    Problem pb{};
    pb.Q = static_cast<const float*>(Qd);
    pb.C = static_cast<const float*>(Cd);
    pb.M = M;
    pb.N = N;
    pb.d = d;
    pb.k = k;
    pb.m = opt.rerank_extra;
    pb.graph = graph;
    pb.thr = static_cast<const float*>(Td);
    pb.out_idx = static_cast<int32_t*>(oi);
    pb.out_dist = static_cast<float*>(od);
    pb.slab_bytes = opt.max_workspace_bytes > 0 ? opt.max_workspace_bytes / 2 : 0;
    pb.precision = opt.precision;
    pb.fused = opt.fused;
    pb.flags = opt.flags;
    knn_stats local{};
    knn_stats* stats = opt.stats ? opt.stats : &local;
    std::memset(stats, 0, sizeof(*stats));
    KNN_TRY(run_problem(pb, stats, st));
    KNN_TRY(sg.copy_back(st));
    return KNN_OK;
}

// Device buffers owned by one call (released when the call returns; calls are synchronous).
struct CallBuffers {
    std::vector<void*> ptrs;
    ~CallBuffers() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    int take(size_t n, T** out) {
        void* p = nullptr;
        const size_t bytes = std::max<size_t>(n * sizeof(T), 16);
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(KNN_ENOMEM, "similarity buffers (%zu bytes): %s", bytes, cudaGetErrorString(e));
        }
        ptrs.push_back(p);
        *out = static_cast<T*>(p);
        return KNN_OK;
    }
};

// Cosine or Pearson similarity search / graph (Methods, "Distance calculation"): unit rows
// in FP32, the k + m nearest unit rows by the Euclidean engine, the FP64 similarity of those
// candidates from the original rows with a certificate, and FP64 over the whole corpus for
// the rows the certificate does not cover.
int metric_impl(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k, int32_t metric,
                int32_t* out_idx, float* out_val, const knn_options* opt_in, bool graph) {
    if (metric == KNN_METRIC_EUCLIDEAN) return search_impl(Q, M, C, N, d, k, out_idx, out_val, opt_in, graph);
    g_last_error.clear();
    if (metric != KNN_METRIC_COSINE && metric != KNN_METRIC_PEARSON)
        return set_error(KNN_EINVAL, "unknown metric %d", metric);
    const knn_options opt = opt_in ? *opt_in : defaults();
    if (opt.row_threshold) return set_error(KNN_EINVAL, "row_threshold applies to the Euclidean metric only");
    KNN_TRY(validate_args(Q, M, C, N, d, k, out_idx, out_val, opt, graph));
    if (M == 0) return KNN_OK;
    const int32_t centered = metric == KNN_METRIC_PEARSON ? 1 : 0;
    cudaStream_t st = stream_of(&opt);
    const auto t0 = std::chrono::steady_clock::now();
    Staged sg;
    const void *Qd = nullptr, *Cd = nullptr;
    KNN_TRY(sg.in(C, static_cast<size_t>(N) * d * sizeof(float), st, &Cd));
    if (graph) {
        Qd = Cd;
    } else {
        KNN_TRY(sg.in(Q, static_cast<size_t>(M) * d * sizeof(float), st, &Qd));
    }
    void *oi = nullptr, *ov = nullptr;
    KNN_TRY(sg.out(out_idx, static_cast<size_t>(M) * k * sizeof(int32_t), &oi));
    KNN_TRY(sg.out(out_val, static_cast<size_t>(M) * k * sizeof(float), &ov));
    const int64_t avail = N - (graph ? 1 : 0);
    const int32_t extra = std::max(opt.rerank_extra, 16);
    const int32_t kp = static_cast<int32_t>(std::min<int64_t>({static_cast<int64_t>(k) + extra, avail, MAX_K}));
    CallBuffers cb;
    float *Uc = nullptr, *Uq = nullptr, *cand_dist = nullptr;
    double *cm = nullptr, *cn = nullptr, *qm = nullptr, *qn = nullptr;
    int32_t *bad = nullptr, *cand_idx = nullptr;
    uint32_t* unc = nullptr;
    KNN_TRY(cb.take(static_cast<size_t>(N) * d, &Uc));
    KNN_TRY(cb.take(static_cast<size_t>(N), &cm));
    KNN_TRY(cb.take(static_cast<size_t>(N), &cn));
    if (graph) {
        Uq = Uc;
        qm = cm;
        qn = cn;
    } else {
        KNN_TRY(cb.take(static_cast<size_t>(M) * d, &Uq));
        KNN_TRY(cb.take(static_cast<size_t>(M), &qm));
        KNN_TRY(cb.take(static_cast<size_t>(M), &qn));
    }
    KNN_TRY(cb.take(1, &bad));
    KNN_TRY(cb.take(static_cast<size_t>(M) * kp, &cand_idx));
    KNN_TRY(cb.take(static_cast<size_t>(M) * kp, &cand_dist));
    KNN_TRY(cb.take(static_cast<size_t>(M), &unc));
    int64_t launches = 0;
    KNN_CK(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
    KNN_CK(launch_sim_prep(static_cast<const float*>(Cd), N, d, centered, Uc, cm, cn, bad, st));
    ++launches;
    if (!graph) {
        KNN_CK(launch_sim_prep(static_cast<const float*>(Qd), M, d, centered, Uq, qm, qn, bad, st));
        ++launches;
    }
    int32_t hbad = 0;
    KNN_CK(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaStreamSynchronize(st));
    if (hbad)
        return set_error(KNN_EINVAL, "a row has zero norm%s or a non-finite value: its similarity is undefined",
                         centered ? " after centring" : "");
    // the nearest unit rows
    Problem pb{};
    pb.Q = Uq;
    pb.C = Uc;
    pb.M = M;
    pb.N = N;
    pb.d = d;
    pb.k = kp;
    pb.m = opt.rerank_extra;
    pb.graph = graph;
    pb.out_idx = cand_idx;
    pb.out_dist = cand_dist;
    pb.slab_bytes = opt.max_workspace_bytes > 0 ? opt.max_workspace_bytes / 2 : 0;
    pb.precision = opt.precision;
    pb.fused = opt.fused;
    pb.flags = opt.flags & ~KNN_FLAG_TIMING;
    knn_stats local{};
    knn_stats* stats = opt.stats ? opt.stats : &local;
    std::memset(stats, 0, sizeof(*stats));
    KNN_TRY(run_problem(pb, stats, st));
    launches += stats->kernel_launches;
    // FP64 similarity of the candidates, certificate
    SimRerankParams rp{};
    rp.Q = static_cast<const float*>(Qd);
    rp.C = static_cast<const float*>(Cd);
    rp.qmean = qm;
    rp.qnorm = qn;
    rp.cmean = cm;
    rp.cnorm = cn;
    rp.cand_idx = cand_idx;
    rp.cand_dist = cand_dist;
    rp.M = M;
    rp.d = d;
    rp.k = k;
    rp.kp = kp;
    rp.P = 32;
    while (rp.P < kp) rp.P *= 2;
    rp.all_candidates = kp == avail ? 1 : 0;
    rp.margin = sim_margin(d);
    rp.out_idx = static_cast<int32_t*>(oi);
    rp.out_val = static_cast<float*>(ov);
    rp.uncertified = unc;
    KNN_CK(launch_sim_rerank(rp, centered, st));
    ++launches;
    std::vector<uint32_t> hu(static_cast<size_t>(M));
    KNN_CK(cudaMemcpyAsync(hu.data(), unc, M * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaStreamSynchronize(st));
    std::vector<int32_t> rows;
    for (int64_t i = 0; i < M; ++i)
        if (hu[static_cast<size_t>(i)]) rows.push_back(static_cast<int32_t>(i));
    stats->rows_uncertified = static_cast<int64_t>(rows.size());
    if (!rows.empty() && !(opt.flags & KNN_FLAG_NO_FALLBACK)) {
        // FP64 over the whole corpus, in batches whose scratch stays within 1 GiB
        const int64_t per = std::max<int64_t>(1, std::min<int64_t>(static_cast<int64_t>(rows.size()),
                                                                   (int64_t(1) << 27) / N));
        int32_t* drows = nullptr;
        double* scratch = nullptr;
        KNN_TRY(cb.take(rows.size(), &drows));
        KNN_TRY(cb.take(static_cast<size_t>(per) * N, &scratch));
        KNN_CK(cudaMemcpyAsync(drows, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        for (int64_t r0 = 0; r0 < static_cast<int64_t>(rows.size()); r0 += per) {
            const int32_t nb = static_cast<int32_t>(std::min<int64_t>(per, static_cast<int64_t>(rows.size()) - r0));
            KNN_CK(launch_exact_rows_sim_fp64(static_cast<const float*>(Qd), static_cast<const float*>(Cd), N, d, k,
                                              graph ? 1 : 0, centered, qm, qn, cm, cn, drows + r0, nb, scratch,
                                              static_cast<int32_t*>(oi), static_cast<float*>(ov), st));
            ++launches;
        }
        stats->rows_fallback += static_cast<int64_t>(rows.size());
    }
    KNN_TRY(sg.copy_back(st));
    KNN_CK(cudaStreamSynchronize(st));
    stats->rows = M;
    stats->kernel_launches = launches;
    if (opt.flags & KNN_FLAG_TIMING)
        stats->ms_total = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return KNN_OK;
}

// k-NN search against a corpus read in chunks (out-of-core): chunk c + 1 is copied on a second
// stream while chunk c is searched; each chunk's exact answer is merged into the running
// answer by (FP64 distance, global index) while the chunk is resident, and the reported
// distances are the FP32 rounding of those FP64 distances.
int stream_impl(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k, int64_t chunk_rows,
                int32_t* out_idx, float* out_dist, const knn_options* opt_in) {
    g_last_error.clear();
    const knn_options opt = opt_in ? *opt_in : defaults();
    if (opt.row_threshold) return set_error(KNN_EINVAL, "row_threshold is not supported with a streamed corpus");
    KNN_TRY(validate_args(Q, M, C, N, d, k, out_idx, out_dist, opt, false));
    if (chunk_rows < 0) return set_error(KNN_EINVAL, "chunk_rows must be >= 0");
    if (M == 0) return KNN_OK;
    cudaStream_t st = stream_of(&opt);
    const auto t0 = std::chrono::steady_clock::now();
    Staged sg;
    const void* Qd = nullptr;
    KNN_TRY(sg.in(Q, static_cast<size_t>(M) * d * sizeof(float), st, &Qd));
    void *oi = nullptr, *od = nullptr;
    KNN_TRY(sg.out(out_idx, static_cast<size_t>(M) * k * sizeof(int32_t), &oi));
    KNN_TRY(sg.out(out_dist, static_cast<size_t>(M) * k * sizeof(float), &od));
    if (chunk_rows == 0) {
        // two chunk buffers in a quarter of the free device memory
        size_t free_b = 0, total_b = 0;
        KNN_CK(cudaMemGetInfo(&free_b, &total_b));
        chunk_rows = static_cast<int64_t>(free_b / 4) / (2 * static_cast<int64_t>(d) * 4);
    }
    chunk_rows = std::max<int64_t>(1, std::min(chunk_rows, N));
    const int32_t kc_max = static_cast<int32_t>(std::min<int64_t>(k, chunk_rows));
    CallBuffers cb;
    float* buf[2] = {nullptr, nullptr};
    KNN_TRY(cb.take(static_cast<size_t>(chunk_rows) * d, &buf[0]));
    if (chunk_rows < N) KNN_TRY(cb.take(static_cast<size_t>(chunk_rows) * d, &buf[1]));
    int32_t *run_idx = nullptr, *cidx = nullptr;
    double* run_d64 = nullptr;
    float *run_f32 = nullptr, *cdist = nullptr;
    KNN_TRY(cb.take(static_cast<size_t>(M) * k, &run_idx));
    KNN_TRY(cb.take(static_cast<size_t>(M) * k, &run_d64));
    KNN_TRY(cb.take(static_cast<size_t>(M) * k, &run_f32));
    KNN_TRY(cb.take(static_cast<size_t>(M) * kc_max, &cidx));
    KNN_TRY(cb.take(static_cast<size_t>(M) * kc_max, &cdist));
    // from the second chunk on, each query's running k-th distance bounds the chunk's search
    // (KNN_STREAM_BOUND=0: every chunk searched without it)
    const char* bound_env = std::getenv("KNN_STREAM_BOUND");
    const bool bound_on = !(bound_env && bound_env[0] == '0');
    float* thr_run = nullptr;
    if (bound_on) KNN_TRY(cb.take(static_cast<size_t>(M), &thr_run));
    struct StreamEvents {
        cudaStream_t cs = nullptr;
        cudaEvent_t copied[2] = {nullptr, nullptr}, merged[2] = {nullptr, nullptr};
        ~StreamEvents() {
            if (cs) cudaStreamSynchronize(cs);
            for (auto e : copied)
                if (e) cudaEventDestroy(e);
            for (auto e : merged)
                if (e) cudaEventDestroy(e);
            if (cs) cudaStreamDestroy(cs);
        }
    } se;
    KNN_CK(cudaStreamCreateWithFlags(&se.cs, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        KNN_CK(cudaEventCreateWithFlags(&se.copied[b], cudaEventDisableTiming));
        KNN_CK(cudaEventCreateWithFlags(&se.merged[b], cudaEventDisableTiming));
    }
    KNN_CK(launch_stream_init(M * k, run_idx, run_d64, run_f32, st));
    int64_t launches = 1;
    // the copy into a buffer waits for the merge that last read it
    auto issue_copy = [&](int64_t c0, int b) -> int {
        const int64_t n = std::min(chunk_rows, N - c0);
        KNN_CK(cudaStreamWaitEvent(se.cs, se.merged[b], 0));
        KNN_CK(cudaMemcpyAsync(buf[b], C + c0 * d, static_cast<size_t>(n) * d * sizeof(float), cudaMemcpyDefault,
                               se.cs));
        KNN_CK(cudaEventRecord(se.copied[b], se.cs));
        return KNN_OK;
    };
    knn_stats* stats = opt.stats;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    KNN_TRY(issue_copy(0, 0));
    int64_t ci = 0;
    for (int64_t c0 = 0; c0 < N; c0 += chunk_rows, ++ci) {
        const int b = static_cast<int>(ci & 1);
        const int64_t n = std::min(chunk_rows, N - c0);
        KNN_CK(cudaStreamWaitEvent(st, se.copied[b], 0));
        if (c0 + chunk_rows < N) KNN_TRY(issue_copy(c0 + chunk_rows, b ^ 1));
        const int32_t kcc = static_cast<int32_t>(std::min<int64_t>(k, n));
        Problem pb{};
        pb.Q = static_cast<const float*>(Qd);
        pb.C = buf[b];
        pb.M = M;
        pb.N = n;
        pb.d = d;
        pb.k = kcc;
        pb.m = opt.rerank_extra;
        pb.graph = false;
        pb.out_idx = cidx;
        pb.out_dist = cdist;
        pb.slab_bytes = opt.max_workspace_bytes > 0 ? opt.max_workspace_bytes / 2 : 0;
        pb.precision = opt.precision;
        pb.fused = opt.fused;
        pb.flags = opt.flags & ~KNN_FLAG_TIMING;
        if (bound_on && ci > 0) {
            KNN_CK(launch_stream_bound(run_d64, M, k, thr_run, st));
            pb.thr = thr_run;
            pb.thr_bound = true;
            ++launches;
        }
        knn_stats cs_stats{};
        KNN_TRY(run_problem(pb, &cs_stats, st));
        StreamMergeParams mp{};
        mp.Q = static_cast<const float*>(Qd);
        mp.chunk = buf[b];
        mp.chunk_row0 = c0;
        mp.chunk_idx = cidx;
        mp.M = M;
        mp.d = d;
        mp.k = k;
        mp.kc = kcc;
        mp.P = 32;
        while (mp.P < k + kcc) mp.P *= 2;
        mp.run_idx = run_idx;
        mp.run_d64 = run_d64;
        mp.run_f32 = run_f32;
        KNN_CK(launch_stream_merge(mp, st));
        KNN_CK(cudaEventRecord(se.merged[b], st));
        launches += cs_stats.kernel_launches + 1;
        if (stats) {
            stats->max_error_ratio = std::max(stats->max_error_ratio, cs_stats.max_error_ratio);
            stats->rows_reranked_in_sweep += cs_stats.rows_reranked_in_sweep;
            stats->candidates += cs_stats.candidates;
            stats->rows_truncated += cs_stats.rows_truncated;
            stats->rows_uncertified += cs_stats.rows_uncertified;
            stats->rows_fallback += cs_stats.rows_fallback;
            stats->rows_fp64_ties += cs_stats.rows_fp64_ties;
            stats->gemm_flops += cs_stats.gemm_flops;
            stats->precision_used = cs_stats.precision_used;
            stats->fused_used = cs_stats.fused_used;
        }
    }
    KNN_CK(cudaMemcpyAsync(oi, run_idx, static_cast<size_t>(M) * k * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    KNN_CK(cudaMemcpyAsync(od, run_f32, static_cast<size_t>(M) * k * sizeof(float), cudaMemcpyDeviceToDevice, st));
    KNN_TRY(sg.copy_back(st));
    KNN_CK(cudaStreamSynchronize(st));
    if (stats) {
        stats->rows = M;
        stats->kernel_launches = launches;
        stats->gemm_launches = static_cast<int32_t>(ci);
        if (opt.flags & KNN_FLAG_TIMING)
            stats->ms_total = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return KNN_OK;
}

// The k smallest of every row of D (M x N, row stride ldd) as sorted (index, value) pairs, and
// each row's RowFlag bits in flags. Few long dense rows are split into S segments selected in
// parallel (one warp per row would leave most SMs idle), whose S k answers are merged: by one
// warp-wide sort when S k <= 1024, else by a select over their concatenation (itself split
// again when it is long) and an index remap. With a sizing arena (ar.sizing()) only the
// workspace is taken and nothing is launched.
int select_rows(const float* D, int64_t M, int64_t N, int64_t ldd, int32_t k, int32_t* oi, float* ov,
                uint32_t* flags, Arena& ar, cudaStream_t st, int64_t* launches) {
    const bool run = !ar.sizing();
    const int S = select_split_segments(M, N, ldd, k, D);
    if (S == 1) {
        if (!run) return KNN_OK;
        SelectParams sp{};
        sp.D = D;
        sp.ldd = ldd;
        sp.M = M;
        sp.N = N;
        sp.spec = select_spec(N);
        sp.block = select_prefers_block(M, k) ? 1 : 0;
        sp.k = k;
        sp.km = k;
        sp.cap = k;
        sp.flags = flags;
        KNN_CK(launch_select_topk(sp, oi, ov, st));
        ++*launches;
        return KNN_OK;
    }
    const int64_t L = N / S, rows = M * S, width = static_cast<int64_t>(S) * k;
    uint32_t* seg_flags = ar.take<uint32_t>(rows);
    int32_t* seg_idx = ar.take<int32_t>(rows * k);
    float* seg_val = ar.take<float>(rows * k);
    int32_t* merged_col = width > 1024 ? ar.take<int32_t>(M * k) : nullptr;
    if (run) {
        SelectParams sp{};
        sp.D = D;
        sp.ldd = L;
        sp.M = rows;
        sp.N = L;
        sp.spec = select_spec(L);
        sp.block = select_prefers_block(M, k) ? 1 : 0;
        sp.k = k;
        sp.km = k;
        sp.cap = k;
        sp.flags = seg_flags;
        KNN_CK(launch_select_topk(sp, seg_idx, seg_val, st));
        ++*launches;
    }
    if (width <= 1024) {
        if (run) {
            KNN_CK(launch_select_merge(seg_idx, seg_val, seg_flags, M, S, k, L, oi, ov, flags, st));
            ++*launches;
        }
        return KNN_OK;
    }
    KNN_TRY(select_rows(seg_val, M, width, width, k, merged_col, ov, flags, ar, st, launches));
    if (run) {
        KNN_CK(launch_select_remap(merged_col, seg_idx, seg_flags, M, S, k, L, oi, flags, st));
        ++*launches;
    }
    return KNN_OK;
}

}  // namespace

// Recomputes the given query rows of pb exactly (the plain FP32 form over gathered rows,
// then FP64 for any it cannot certify), writing their output rows in place: the
// fallback of the batched form for rows its re-rank could not certify.
int recompute_rows(const Problem& pb, const std::vector<int32_t>& rows, cudaStream_t st) {
    if (rows.empty()) return KNN_OK;
    CommonLayout L;
    {
        Arena sz;
        layout_common(pb, P_FP32, true, sz, L);
        void* base = nullptr;
        KNN_TRY(workspace_get(sz.used(), &base));
        Arena ar(static_cast<char*>(base), sz.used());
        L = CommonLayout{};
        layout_common(pb, P_FP32, true, ar, L);
    }
    Timing tm;
    KNN_TRY(prep_and_check(pb, P_FP32, L, st, nullptr, tm));
    KNN_CK(cudaMemsetAsync(L.counters, 0, sizeof(RerankCounters), st));
    int64_t n64 = 0;
    KNN_TRY(plain_fallback(pb, L, rows, st, tm, &n64));
    KNN_CK(cudaStreamSynchronize(st));
    return KNN_OK;
}


int run_problem(const Problem& pb, knn_stats* stats, cudaStream_t st) {
    int prec = pb.precision;
    const int km = static_cast<int>(std::min<int64_t>(pb.k + pb.m, pb.N - (pb.graph ? 1 : 0)));
    const int want = prec == KNN_FP8_E4M3 ? P_FP8 : P_BF16;
    const bool fused_ok = fused_available() && fused_stages(fused_cap(pb.k, km), want) > 0 && pb.fused != 0;
    if (prec == KNN_AUTO) prec = fused_ok ? KNN_BF16 : KNN_FP32;
    switch (prec) {
        case KNN_FP32:
            if (pb.fused == 1) return set_error(KNN_EUNSUPPORTED, "the FP32 form is not fused");
            return run_plain(pb, stats, st);
        case KNN_BF16:
        case KNN_FP8_E4M3:
            if (!fused_ok)
                return set_error(KNN_EUNSUPPORTED,
                                 "the tensor-core form needs an sm_103 device and k + m small enough for its "
                                 "shared-memory candidate buffers; got k=%d m=%d", pb.k, pb.m);
            return run_fused(pb, prec == KNN_BF16 ? P_BF16 : P_FP8, stats, st);
        default:
            return set_error(KNN_EINVAL, "unknown precision %d", prec);
    }
}

}  // namespace knn

// ---------------------------------------------------------------------------
// extern "C" surface
// ---------------------------------------------------------------------------
extern "C" {

void knn_options_init(knn_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = KNN_AUTO;
    opt->rerank_extra = 32;
    opt->fused = -1;
    opt->flags = KNN_FLAG_CHECK_FINITE;
}

int knng_build(const float* X, int64_t N, int32_t d, int32_t k, int32_t* out_idx, float* out_dist) {
    return knn::search_impl(X, N, X, N, d, k, out_idx, out_dist, nullptr, true);
}

int knng_build_ex(const float* X, int64_t N, int32_t d, int32_t k, int32_t* out_idx, float* out_dist,
                  const knn_options* opt) {
    return knn::search_impl(X, N, X, N, d, k, out_idx, out_dist, opt, true);
}

int knn_search(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k, int32_t* out_idx,
               float* out_dist, const knn_options* opt) {
    return knn::search_impl(Q, M, C, N, d, k, out_idx, out_dist, opt, false);
}

int knn_search_metric(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k, int32_t metric,
                      int32_t* out_idx, float* out_val, const knn_options* opt) {
    return knn::metric_impl(Q, M, C, N, d, k, metric, out_idx, out_val, opt, false);
}

int knng_build_metric(const float* X, int64_t N, int32_t d, int32_t k, int32_t metric, int32_t* out_idx,
                      float* out_val, const knn_options* opt) {
    return knn::metric_impl(X, N, X, N, d, k, metric, out_idx, out_val, opt, true);
}

int knn_search_streamed(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k,
                        int64_t chunk_rows, int32_t* out_idx, float* out_dist, const knn_options* opt) {
    return knn::stream_impl(Q, M, C, N, d, k, chunk_rows, out_idx, out_dist, opt);
}

int knn_select(const float* D, int64_t M, int64_t N, int64_t ldd, int32_t k, int32_t* out_idx, float* out_val,
               const knn_options* opt) {
    using namespace knn;
    g_last_error.clear();
    if (!D || !out_idx || !out_val) return set_error(KNN_EINVAL, "NULL pointer argument");
    if (N < 1 || N >= (int64_t(1) << 31)) return set_error(KNN_EINVAL, "N must be in [1, 2^31)");
    if (ldd < N) return set_error(KNN_EINVAL, "ldd (%lld) must be >= N (%lld)", (long long)ldd, (long long)N);
    if (k < 1 || k > N) return set_error(KNN_EINVAL, "k must be in [1, N] (k=%d, N=%lld)", k, (long long)N);
    if (k > MAX_K) return set_error(KNN_EINVAL, "k above %d is not supported", MAX_K);
    if (M < 0) return set_error(KNN_EINVAL, "M must be >= 0");
    if (M == 0) return KNN_OK;
    cudaStream_t st = stream_of(opt);
    Staged sg;
    const void* Dd = nullptr;
    KNN_TRY(sg.in(D, (static_cast<size_t>(M - 1) * ldd + N) * sizeof(float), st, &Dd));
    void *oi = nullptr, *ov = nullptr;
    KNN_TRY(sg.out(out_idx, static_cast<size_t>(M) * k * sizeof(int32_t), &oi));
    KNN_TRY(sg.out(out_val, static_cast<size_t>(M) * k * sizeof(float), &ov));
    knn_stats* stats = opt ? opt->stats : nullptr;
    const bool timing = stats && (opt->flags & KNN_FLAG_TIMING);
    const auto t0 = std::chrono::steady_clock::now();
    uint32_t* flags = nullptr;
    int64_t launches = 0;
    Arena sz;
    flags = sz.take<uint32_t>(M);
    KNN_TRY(select_rows(static_cast<const float*>(Dd), M, N, ldd, k, nullptr, nullptr, flags, sz, st, &launches));
    void* base = nullptr;
    KNN_TRY(workspace_get(sz.used(), &base));
    Arena ar(static_cast<char*>(base), sz.used());
    flags = ar.take<uint32_t>(M);
    Events ev;
    KNN_TRY(ev.init(timing));
    KNN_TRY(ev.rec(0, st));
    launches = 0;
    KNN_TRY(select_rows(static_cast<const float*>(Dd), M, N, ldd, k, static_cast<int32_t*>(oi), static_cast<float*>(ov),
                        flags, ar, st, &launches));
    KNN_TRY(ev.rec(1, st));
    std::vector<uint32_t> hf(static_cast<size_t>(M));
    KNN_CK(cudaMemcpyAsync(hf.data(), flags, M * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < M; ++i)
        if (hf[static_cast<size_t>(i)] & ROW_SELECT_ERROR)
            return set_error(KNN_EINVAL, "row %lld holds NaN (or the select gave up)", (long long)i);
    KNN_TRY(sg.copy_back(st));
    if (stats) {
        *stats = knn_stats{};
        stats->rows = M;
        stats->kernel_launches = launches;
        if (timing) {
            KNN_CK(cudaEventElapsedTime(&stats->ms_select, ev.ev[0], ev.ev[1]));
            stats->ms_total =
                std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
    }
    return KNN_OK;
}

int knn_distances(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, float* out_D, int64_t ldd,
                  int32_t full, const knn_options* opt) {
    using namespace knn;
    g_last_error.clear();
    if (!Q || !C || !out_D) return set_error(KNN_EINVAL, "NULL pointer argument");
    if (d < 1 || N < 1 || M < 0) return set_error(KNN_EINVAL, "bad sizes");
    if (ldd < N) return set_error(KNN_EINVAL, "ldd must be >= N");
    if (M == 0) return KNN_OK;
    cudaStream_t st = stream_of(opt);
    Staged sg;
    const void *Qd = nullptr, *Cd = nullptr;
    KNN_TRY(sg.in(Q, static_cast<size_t>(M) * d * sizeof(float), st, &Qd));
    KNN_TRY(sg.in(C, static_cast<size_t>(N) * d * sizeof(float), st, &Cd));
    void* Dd = nullptr;
    KNN_TRY(sg.out(out_D, (static_cast<size_t>(M - 1) * ldd + N) * sizeof(float), &Dd));
    Arena sz;
    sz.take<PrepGlobals>(2);
    sz.take<float>(N);
    sz.take<float>(M);
    void* base = nullptr;
    KNN_TRY(workspace_get(sz.used(), &base));
    Arena ar(static_cast<char*>(base), sz.used());
    PrepGlobals* g = ar.take<PrepGlobals>(2);
    float* cn = ar.take<float>(N);
    float* qn = ar.take<float>(M);
    KNN_CK(cudaMemsetAsync(g, 0, 2 * sizeof(PrepGlobals), st));
    KNN_CK(launch_prep(static_cast<const float*>(Cd), N, d, P_FP32, cn, nullptr, nullptr, nullptr, 0, nullptr, g, st));
    if (full)
        KNN_CK(launch_prep(static_cast<const float*>(Qd), M, d, P_FP32, qn, nullptr, nullptr, nullptr, 0, nullptr,
                           g + 1, st));
    KNN_CK(launch_gemm_simt(static_cast<const float*>(Qd), M, 0, static_cast<const float*>(Cd), N, d, cn,
                            full ? qn : nullptr, static_cast<float*>(Dd), ldd, 0, st));
    KNN_TRY(sg.copy_back(st));
    KNN_CK(cudaStreamSynchronize(st));
    return KNN_OK;
}

int knn_search_batched(knn_problem* probs, int32_t count, const knn_options* opt_in) {
    using namespace knn;
    g_last_error.clear();
    if (count < 0 || (count > 0 && !probs)) return set_error(KNN_EINVAL, "bad problem list");
    const knn_options opt = opt_in ? *opt_in : defaults();
    cudaStream_t st = stream_of(&opt);
    int first = KNN_OK;
    std::vector<Problem> batch;
    std::vector<int> where;
    for (int32_t i = 0; i < count; ++i) {
        knn_problem& p = probs[i];
        const bool graph = p.exclude_self != 0;
        const float* Q = (graph && !p.Q) ? p.C : p.Q;
        p.status = validate_args(Q, p.M, p.C, p.N, p.d, p.k, p.out_idx, p.out_dist, opt, graph);
        if (p.status == KNN_OK && graph && Q != p.C) p.status = set_error(KNN_EINVAL, "a graph problem needs Q == C");
        if (p.status != KNN_OK) {
            if (first == KNN_OK) first = p.status;
            continue;
        }
        if (p.M == 0) continue;
        const bool device = is_device_pointer(p.C) && is_device_pointer(Q) && is_device_pointer(p.out_idx) &&
                            is_device_pointer(p.out_dist);
        if (!device) {
            // host arrays: the single-problem path stages them
            p.status = search_impl(Q, p.M, p.C, p.N, p.d, p.k, p.out_idx, p.out_dist, &opt, graph);
            if (p.status != KNN_OK && first == KNN_OK) first = p.status;
            continue;
        }
        Problem pb{};
        pb.Q = Q;
        pb.C = p.C;
        pb.M = p.M;
        pb.N = p.N;
        pb.d = p.d;
        pb.k = p.k;
        pb.m = opt.rerank_extra;
        pb.graph = graph;
        pb.out_idx = p.out_idx;
        pb.out_dist = p.out_dist;
        pb.precision = opt.precision;
        pb.fused = opt.fused;
        pb.flags = opt.flags;
        batch.push_back(pb);
        where.push_back(i);
    }
    if (!batch.empty()) {
        std::vector<int> status(batch.size(), KNN_OK);
        knn_stats local{};
        knn_stats* stats = opt.stats ? opt.stats : &local;
        std::memset(stats, 0, sizeof(*stats));
        const int rc = run_batch(batch, status, opt.precision, stats, st);
        for (size_t j = 0; j < batch.size(); ++j) {
            probs[where[j]].status = rc != KNN_OK && status[j] == KNN_OK ? rc : status[j];
            if (probs[where[j]].status != KNN_OK && first == KNN_OK) first = probs[where[j]].status;
        }
        if (rc != KNN_OK && first == KNN_OK) first = rc;
    }
    return first;
}

const char* knn_status_string(int status) {
    switch (status) {
        case KNN_OK: return "KNN_OK";
        case KNN_EINVAL: return "KNN_EINVAL";
        case KNN_ENOMEM: return "KNN_ENOMEM";
        case KNN_ECUDA: return "KNN_ECUDA";
        case KNN_ETIMEOUT: return "KNN_ETIMEOUT";
        case KNN_EINTERNAL: return "KNN_EINTERNAL";
        case KNN_EUNSUPPORTED: return "KNN_EUNSUPPORTED";
        default: return "KNN_UNKNOWN";
    }
}

const char* knn_last_error(void) { return knn::g_last_error.c_str(); }

void knn_shutdown(void) { knn::workspace_release_all(); }

const char* knn_version(void) { return "0.1.0"; }

}  // extern "C"
