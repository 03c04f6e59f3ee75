// Host-side runtime structures of the engine (internal; not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"
#include "knn.h"

namespace knn {

constexpr int MAX_CAP = 2048;  // largest candidate list per row
constexpr int MAX_K = 1024;

extern thread_local std::string g_last_error;
int set_error(int status, const char* fmt, ...);

#define KNN_CK(expr)                                                                                   \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            return ::knn::set_error(-3, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                                    __LINE__);                                                         \
        }                                                                                              \
    } while (0)

#define KNN_TRY(expr)          \
    do {                       \
        int s_ = (expr);       \
        if (s_ != 0) return s_; \
    } while (0)

// Bump allocator over the workspace. With base == nullptr it only measures.
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    Arena() = default;
    Arena(char* b, size_t c) : base(b), cap(c) {}
    bool sizing() const { return base == nullptr; }
    size_t used() const { return off; }
    template <typename T>
    T* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

// One k-NN problem with device pointers.
struct Problem {
    const float* Q;
    const float* C;
    int64_t M, N;
    int32_t d, k, m;
    bool graph;           // k-NN graph: Q == C, row i excludes column i
    const float* thr;     // optional per-row squared-distance thresholds (device), M entries
    // thr bounds the answer instead of guessing it (the out-of-core search's running k-th
    // distance): a point farther than thr[i] is not wanted, a row may keep fewer than k points,
    // and its answer is exact among the points at or below thr[i]
    bool thr_bound = false;
    int32_t* out_idx;     // M x k
    float* out_dist;      // M x k
    int64_t slab_bytes;   // distance-matrix slab budget (0 = default)
    int32_t precision;    // Precision
    int32_t fused;        // -1 auto, 0, 1
    int32_t flags;        // KNN_FLAG_*
    int32_t spec = -1;    // speculative thresholds in the fused sweep: -1 by the size rule, 0 off, 1 on
    int32_t sched = -1;   // batched form: the schedule to take (the autotuner's timing runs), -1: chosen
};

struct PrepState {
    PrepGlobals* gq;
    PrepGlobals* gc;
    float* qnorm2;
    float* cnorm2;
    float* qres;
    float* cres;
    float* qtn;
    float* ctn;
    float* E;
    float* thr_dprime;  // per-row threshold converted to d' scale (or nullptr)
    void* xq;           // reduced-precision queries (graph: shared with xc)
    void* xc;
    float* qscale;
    float* cscale;
    int32_t d_pad;
};

// The library's cached device workspace (grow-only). A call running under a
// WorkspaceCap fails with KNN_ENOMEM instead of growing it past the cap.
int workspace_get(size_t bytes, void** out);
struct WorkspaceCap {
    explicit WorkspaceCap(int64_t bytes);  // 0: no cap
    ~WorkspaceCap();
    WorkspaceCap(const WorkspaceCap&) = delete;
    WorkspaceCap& operator=(const WorkspaceCap&) = delete;

   private:
    int64_t prev_;
};
void workspace_release_all();
bool is_device_pointer(const void* p);
int pick_cap(int k, int km);

cudaError_t launch_select_ex(const SelectParams& p, int64_t self_offset, bool check_nan, cudaStream_t st);
cudaError_t launch_threshold_to_dprime(const float* thr, const float* qnorm2, int64_t M, float* out, cudaStream_t st);
// Bounding thresholds (squared distances) to the d' scale of the approximate values: every point
// whose exact squared distance is at most thr[i] has an approximate value at most out[i] (the
// row's bound E[i] and the FP32 roundings of |q|^2 added); non-finite or negative entries: none.
cudaError_t launch_bound_to_dprime(const float* thr, const float* qnorm2, const float* E, int64_t M, int32_t d,
                                   float* out, cudaStream_t st);
cudaError_t launch_gather_rows(const float* Q, int32_t d, const int32_t* rows, int32_t n, const float* E,
                               const float* thr, float* Qs, float* Es, float* Ts, cudaStream_t st);
// Gathers rows of a reduced-precision operand (row_bytes a multiple of 16) and, when
// qscale is given, their scales.
cudaError_t launch_gather_qrows(const void* xq, int32_t row_bytes, const float* qscale, const int32_t* rows, int32_t n,
                                void* out, float* out_scale, cudaStream_t st);
cudaError_t launch_scatter_out(const int32_t* rows, int32_t n, int32_t k, const int32_t* oi_s, const float* od_s,
                               int32_t* oi, float* od, cudaStream_t st);

// Runs one problem end to end (device pointers); fills stats when non-null.
int run_problem(const Problem& pb, ::knn_stats* stats, cudaStream_t st);
// Exact recomputation of the given query rows of pb in place (plain FP32 form, then FP64).
int recompute_rows(const Problem& pb, const std::vector<int32_t>& rows, cudaStream_t st);

// Runs independent problems (device pointers) as one batch: one CUDA graph holding a
// persistent fused launch and the plain form's launches. status[i] receives each
// problem's status; returns the first failure.
int run_batch(std::vector<Problem>& probs, std::vector<int>& status, int precision_req, ::knn_stats* stats,
              cudaStream_t st);

}  // namespace knn
