// knn_select_noalloc: the quick multi-select for callers that must not allocate.
//
// Some callers cannot let a library call cudaMalloc: applications whose device memory
// is all owned by their own caching allocator or by a pool reserved at start-up (a
// library allocation there can fail, or fragment memory the application has already
// planned), and latency-critical paths that cannot pay cudaMalloc's implicit device
// synchronisation in the middle of their work. This entry point serves them: it uses
// no library workspace and stages nothing, so it calls no cudaMalloc, cudaFree or other
// allocating routine. Its only scratch -- one status word per row plus an error
// summary -- is a file-scope device array of fixed size, which every GPU that loads
// the library holds until the process exits.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it. Every later call
// reuses the same array, so calls that overlap on the GPU (different streams, or host
// threads without ordering) race on it and must be serialised by the caller. Like the
// library's other calls it is synchronous: it ends by copying the error summary to a
// host variable and synchronising the stream.
//
// Few long rows are not split into segments here (knn_select does that, with workspace
// for the segment answers): for at most 64 rows the select takes one CTA per row, which
// is slower than knn_select's split when the rows are very long.
#include <cuda_runtime.h>

#include <mutex>

#include "engine.h"
#include "internal.h"
#include "knn.h"

namespace knn {
namespace {

// Maximum rows per call (4 MiB of status words).
constexpr int64_t NOALLOC_MAX_ROWS = int64_t(1) << 20;
constexpr int NOALLOC_MAX_DEVICES = 64;

struct NoallocScratch {
    uint32_t row_flags[NOALLOC_MAX_ROWS];  // RowFlag bits of every row of the last call
    uint32_t any_error;                    // OR of row_flags & ROW_SELECT_ERROR (cleared per call)
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

std::mutex g_noalloc_mu;
NoallocScratch* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per device).
int noalloc_scratch(NoallocScratch** out) {
    int dev = 0;
    KNN_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return set_error(KNN_EUNSUPPORTED, "device ordinal %d too large", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(KNN_ECUDA, "cudaGetSymbolAddress of the select scratch failed: %s",
                             cudaGetErrorString(e));
        }
        g_noalloc_ptr[dev] = static_cast<NoallocScratch*>(ptr);
    }
    *out = g_noalloc_ptr[dev];
    return KNN_OK;
}

// ORs the error bit of every row's status into any_error (device code names the array).
__global__ void noalloc_error_summary(int64_t M) {
    uint32_t e = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < M;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        e |= g_noalloc_scratch.row_flags[i] & ROW_SELECT_ERROR;
    e = __reduce_or_sync(0xffffffffu, e);
    if ((threadIdx.x & 31u) == 0 && e) atomicOr(&g_noalloc_scratch.any_error, e);
}

}  // namespace
}  // namespace knn

extern "C" int knn_select_noalloc(const float* D, int64_t M, int64_t N, int64_t ldd, int32_t k, int32_t* out_idx,
                                  float* out_val, void* stream) {
    using namespace knn;
    g_last_error.clear();
    if (!D || !out_idx || !out_val) return set_error(KNN_EINVAL, "NULL pointer argument");
    if (N < 1 || N >= (int64_t(1) << 31)) return set_error(KNN_EINVAL, "N must be in [1, 2^31)");
    if (ldd < N) return set_error(KNN_EINVAL, "ldd (%lld) must be >= N (%lld)", (long long)ldd, (long long)N);
    if (k < 1 || k > N) return set_error(KNN_EINVAL, "k must be in [1, N] (k=%d, N=%lld)", k, (long long)N);
    if (k > MAX_K) return set_error(KNN_EINVAL, "k above %d is not supported", MAX_K);
    if (M < 0) return set_error(KNN_EINVAL, "M must be >= 0");
    if (M > NOALLOC_MAX_ROWS)
        return set_error(KNN_EINVAL, "knn_select_noalloc handles at most %lld rows per call (got %lld)",
                         (long long)NOALLOC_MAX_ROWS, (long long)M);
    if (!is_device_pointer(D) || !is_device_pointer(out_idx) || !is_device_pointer(out_val))
        return set_error(KNN_EINVAL, "knn_select_noalloc takes device pointers only (it stages nothing)");
    if (M == 0) return KNN_OK;
    NoallocScratch* scratch = nullptr;
    KNN_TRY(noalloc_scratch(&scratch));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    KNN_CK(cudaMemsetAsync(&scratch->any_error, 0, sizeof(uint32_t), st));
    SelectParams sp{};
    sp.D = D;
    sp.ldd = ldd;
    sp.M = M;
    sp.N = N;
    sp.spec = select_spec(sp.N);
    sp.block = select_prefers_block(M, k) ? 1 : 0;
    sp.k = k;
    sp.km = k;
    sp.cap = k;
    sp.flags = scratch->row_flags;  // every row's word is written by the select
    KNN_CK(launch_select_topk(sp, out_idx, out_val, st));
    const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((M + 255) / 256, 1024));
    noalloc_error_summary<<<blocks, 256, 0, st>>>(M);
    KNN_CK(cudaGetLastError());
    uint32_t any_error = 0;
    KNN_CK(cudaMemcpyAsync(&any_error, &scratch->any_error, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaStreamSynchronize(st));
    if (any_error) return set_error(KNN_EINVAL, "a row holds NaN (or the select gave up)");
    return KNN_OK;
}
