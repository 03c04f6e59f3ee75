// Many independent k-NN search problems of uneven shape in one CUDA graph: one
// persistent launch of the fused tensor-core kernel over the (problem, row block) work
// items of every problem the autotuner assigns to it, batched prep / bounds / re-rank
// kernels over all rows of all problems, and the plain FP32 form (SIMT GEMM slab ->
// quick multi-select -> re-rank) for the problems assigned to it (those whose k + m
// exceed the fused kernel's shared-memory lists, or that the autotuner found faster
// there).
//
// Paper: Methods (coarse-level parallelism: independent queries processed in parallel)
// and Results (kernel launch overhead; the saturation of the GPU needs enough rows).
// One graph replays the whole batch with a single host submission; within it, one
// persistent kernel lets the small problems share the 152 SMs instead of each leaving
// most of them idle.
#include <cuda_runtime.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "engine.h"
#include "internal.h"
#include "knn.h"
#include "tc_fused.h"

namespace knn {

// Schedules a problem of a batch can take: the fused tensor-core form on 128 x 256 tiles (one
// CTA an SM) or on 128 x 128 tiles (two CTAs an SM: twice the epilogue warps per SM, for lists
// of at most 512 keys), each with speculative thresholds in its sweep or without them (a
// choice of the select's work inside the GEMM epilogue), or the plain FP32 form (SIMT GEMM
// slabs, unfused multi-select). SCHED_FUSED leaves speculation to the size rule (from 16384
// points on).
enum Schedule : int {
    SCHED_FUSED = 0,
    SCHED_PLAIN = 1,
    SCHED_FUSED_NOSPEC = 2,
    SCHED_FUSED_SPEC = 3,
    SCHED_FUSED_T128_NOSPEC = 4,
    SCHED_FUSED_T128_SPEC = 5,
};
constexpr int SCHED_LAST = SCHED_FUSED_T128_SPEC;
constexpr int TUNE_VERSION = 4;  // bumped when the schedule table or its timing changes

bool is_fused(int sched) { return sched != SCHED_PLAIN; }
// corpus columns of a fused schedule's tiles
int tile_of(int sched) { return sched == SCHED_FUSED_T128_NOSPEC || sched == SCHED_FUSED_T128_SPEC ? 128 : 256; }
// speculative thresholds: 1 on, 0 off, -1 by the size rule
int spec_of(int sched) {
    if (sched == SCHED_FUSED_SPEC || sched == SCHED_FUSED_T128_SPEC) return 1;
    if (sched == SCHED_FUSED_NOSPEC || sched == SCHED_FUSED_T128_NOSPEC) return 0;
    return -1;
}

const char* schedule_name(int sched) {
    switch (sched) {
        case SCHED_PLAIN: return "plain-fp32";
        case SCHED_FUSED_NOSPEC: return "fused-no-speculation";
        case SCHED_FUSED_SPEC: return "fused-speculation";
        case SCHED_FUSED_T128_NOSPEC: return "fused-128-no-speculation";
        case SCHED_FUSED_T128_SPEC: return "fused-128-speculation";
        default: return "fused";
    }
}

namespace {

// --------------------------------------------------------------------------------------
// autotuner: schedule per shape bucket, measured once on a synthetic problem of the
// bucket, cached in a JSON file (KNN_AUTOTUNE_CACHE, default ~/.cache/knn_gb300_autotune.json)
// whose "_device" entry names the GPU, its SM count and the schedule table's version;
// entries written for another device or version are ignored.
// --------------------------------------------------------------------------------------
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string tune_device_tag() {
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    char b[320];
    std::snprintf(b, sizeof(b), "%s sm%d v%d", prop.name, prop.multiProcessorCount, TUNE_VERSION);
    for (char* c = b; *c; ++c)
        if (*c == '"' || *c == '\\') *c = '_';
    return b;
}

std::string tune_path() {
    const char* e = std::getenv("KNN_AUTOTUNE_CACHE");
    if (e && *e) return e;
    const char* h = std::getenv("HOME");
    return std::string(h ? h : "/tmp") + "/.cache/knn_gb300_autotune.json";
}

void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    FILE* f = std::fopen(tune_path().c_str(), "r");
    if (!f) return;
    char key[320];
    // the file is a flat JSON object {"_device": "tag", "bucket": schedule, ...}
    std::map<std::string, int> entries;
    std::string device;
    int c;
    while ((c = std::fgetc(f)) != EOF) {
        if (c != '"') continue;
        int n = 0;
        while ((c = std::fgetc(f)) != EOF && c != '"' && n < 319) key[n++] = static_cast<char>(c);
        key[n] = 0;
        if (std::strcmp(key, "_device") == 0) {
            while ((c = std::fgetc(f)) != EOF && c != '"') {
            }
            std::string tag;
            while ((c = std::fgetc(f)) != EOF && c != '"') tag += static_cast<char>(c);
            device = tag;
            continue;
        }
        int v;
        if (std::fscanf(f, " : %d", &v) == 1 && v >= SCHED_FUSED && v <= SCHED_LAST) entries[key] = v;
    }
    std::fclose(f);
    if (device == tune_device_tag()) g_tune = entries;
}

void tune_save() {
    const std::string path = tune_path();
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos) {
        const std::string dir = path.substr(0, slash);
        std::string cmd_dir = dir;  // create the directory without a shell: mkdir -p equivalent
        for (size_t i = 1; i <= cmd_dir.size(); ++i)
            if (i == cmd_dir.size() || cmd_dir[i] == '/') {
                const std::string part = cmd_dir.substr(0, i);
                (void)::mkdir(part.c_str(), 0755);
            }
    }
    // a temporary file of this process, renamed over the cache (concurrent writers each
    // replace the whole file; the last one wins)
    const std::string tmp = path + "." + std::to_string(static_cast<long long>(::getpid())) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n  \"_device\": \"%s\"%s\n", tune_device_tag().c_str(), g_tune.empty() ? "" : ",");
    size_t i = 0;
    for (const auto& kv : g_tune)
        std::fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++i < g_tune.size() ? "," : "");
    std::fprintf(f, "}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path.c_str());
}

int ilog2(int64_t x) {
    int r = 0;
    while (x > 1) {
        x >>= 1;
        ++r;
    }
    return r;
}

std::string bucket_of(const Problem& p) {
    char b[160];
    const int kc = p.k <= 8 ? 8 : (p.k <= 32 ? 32 : (p.k <= 128 ? 128 : 1024));
    std::snprintf(b, sizeof(b), "d%d_k%d_m%d_n%d_x%d", (p.d + 63) / 64 * 64, kc, p.m, ilog2(p.N), ilog2(p.M));
    return b;
}

__global__ void synth_kernel(float* x, int64_t n, uint64_t seed) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint64_t z = seed + static_cast<uint64_t>(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[i] = static_cast<float>(static_cast<double>(z >> 11) * 0x1p-53) - 0.5f;
    }
}

}  // namespace
int run_batch(std::vector<Problem>& probs, std::vector<int>& status, int precision_req, ::knn_stats* stats,
              cudaStream_t st);
namespace {
void drop_batch_graph(const std::vector<Problem>& probs, const std::vector<int>& sched, int prec);

// Times one schedule on a synthetic problem of p's shape (at most 4096 query rows), as a batch
// of copies of that problem (the path the schedule will run on) with enough row blocks to fill
// every CTA slot of the GPU, so that schedules that share an SM between CTAs are timed as they
// run inside a full batch; ms per row.
int time_schedule(const Problem& p, int sched, float* ms_per_row) {
    const int64_t M = std::min<int64_t>(p.M, 4096);
    int dev = 0, sms = 1;
    KNN_CK(cudaGetDevice(&dev));
    KNN_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t rb = (M + 127) / 128;
    const int copies = static_cast<int>(std::max<int64_t>(1, (2 * static_cast<int64_t>(sms) + rb - 1) / rb));
    float *Q = nullptr, *C = nullptr, *od = nullptr;
    int32_t* oi = nullptr;
    cudaStream_t st = nullptr;
    KNN_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    const size_t out_elems = static_cast<size_t>(M) * p.k * copies;
    cudaError_t e = cudaMalloc(&Q, static_cast<size_t>(M) * p.d * 4);
    if (e == cudaSuccess) e = cudaMalloc(&C, static_cast<size_t>(p.N) * p.d * 4);
    if (e == cudaSuccess) e = cudaMalloc(&oi, out_elems * 4);
    if (e == cudaSuccess) e = cudaMalloc(&od, out_elems * 4);
    int rc = KNN_OK;
    if (e != cudaSuccess) {
        cudaGetLastError();
        rc = set_error(KNN_ENOMEM, "autotuner buffers: %s", cudaGetErrorString(e));
    } else {
        synth_kernel<<<512, 256, 0, st>>>(Q, M * p.d, 7);
        synth_kernel<<<512, 256, 0, st>>>(C, p.N * p.d, 11);
        Problem q = p;
        q.Q = Q;
        q.C = C;
        q.M = M;
        q.graph = false;
        q.thr = nullptr;
        q.flags = KNN_FLAG_NO_FALLBACK;
        q.precision = is_fused(sched) ? KNN_BF16 : KNN_FP32;
        q.fused = is_fused(sched) ? 1 : 0;
        q.spec = spec_of(sched);
        q.sched = sched;
        std::vector<Problem> batch(static_cast<size_t>(copies), q);
        for (int c = 0; c < copies; ++c) {
            batch[c].out_idx = oi + static_cast<size_t>(c) * M * p.k;
            batch[c].out_dist = od + static_cast<size_t>(c) * M * p.k;
        }
        std::vector<int> status(batch.size(), KNN_OK);
        float best = 1e30f;
        for (int rep = 0; rep < 3 && rc == KNN_OK; ++rep) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, st);
            rc = run_batch(batch, status, q.precision, nullptr, st);
            cudaEventRecord(b, st);
            cudaEventSynchronize(b);
            float t = 0.f;
            cudaEventElapsedTime(&t, a, b);
            if (rep > 0) best = std::min(best, t);
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
        *ms_per_row = best / static_cast<float>(M * copies);
        std::vector<int> scheds(batch.size(), sched);
        drop_batch_graph(batch, scheds, P_BF16);
    }
    cudaStreamSynchronize(st);
    cudaFree(Q);
    cudaFree(C);
    cudaFree(oi);
    cudaFree(od);
    cudaStreamDestroy(st);
    return rc;
}

// Schedule of one problem: the plain form when the fused kernel cannot take it,
// otherwise the cached (or freshly measured) faster form of its bucket.
int choose_schedule(const Problem& p, int precision_req, bool* fused_capable) {
    const int km = static_cast<int>(std::min<int64_t>(p.k + p.m, p.N - (p.graph ? 1 : 0)));
    const int want = precision_req == KNN_FP8_E4M3 ? P_FP8 : P_BF16;
    *fused_capable = fused_available() && fused_stages(fused_cap(p.k, km), want) > 0 && p.fused != 0;
    const bool t128 = *fused_capable && fused_stages(fused_cap(p.k, km), want, false, 128) > 0;
    if (p.sched >= 0) {
        // forced (the autotuner's timing runs): kept where the problem can take it
        if (!is_fused(p.sched)) return SCHED_PLAIN;
        if (!*fused_capable) return SCHED_PLAIN;
        return tile_of(p.sched) == 128 && !t128 ? SCHED_FUSED : p.sched;
    }
    if (!*fused_capable || precision_req == KNN_FP32) return SCHED_PLAIN;
    // KNN_BATCH_TILE=128: every problem that can takes the 128-column tiles (tests, tuning)
    if (const char* te = std::getenv("KNN_BATCH_TILE"); te && std::atoi(te) == 128 && t128)
        return p.N >= 16384 ? SCHED_FUSED_T128_SPEC : SCHED_FUSED_T128_NOSPEC;
    if (p.fused == 1 || precision_req != KNN_AUTO) return SCHED_FUSED;
    const char* env = std::getenv("KNN_AUTOTUNE");
    if (env && env[0] == '0') return SCHED_FUSED;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load();
    const std::string key = bucket_of(p);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
    // the fastest schedule per row of the bucket's synthetic problem (speculation needs a
    // sweep of a few tiles: below 512 points only the plain sweep is timed)
    int sched = SCHED_FUSED;
    float best = 1e30f;
    for (int s : {SCHED_FUSED_SPEC, SCHED_FUSED_NOSPEC, SCHED_FUSED_T128_SPEC, SCHED_FUSED_T128_NOSPEC, SCHED_PLAIN}) {
        if (spec_of(s) == 1 && p.N < 512) continue;
        if (tile_of(s) == 128 && (!t128 || !is_fused(s))) continue;
        float t = 0.f;
        if (time_schedule(p, s, &t) == KNN_OK && t < best) {
            best = t;
            sched = s;
        }
    }
    g_last_error.clear();
    g_tune[key] = sched;
    tune_save();
    return sched;
}

// --------------------------------------------------------------------------------------
// batch workspace (separate from the single-call workspace so a cached graph's buffers
// are not moved by other calls) and graph cache
// --------------------------------------------------------------------------------------
struct BatchWs {
    void* ptr = nullptr;
    size_t bytes = 0;
    uint64_t generation = 0;
};
std::mutex g_bws_mu;
std::map<int, BatchWs> g_bws;

// Phase marks recorded inside a batch's graph: start, after prep and bounds, after the
// fused launch, after the fused problems' re-rank, end (after the plain problems).
constexpr int N_MARKS = 5;

struct BatchLayout;

// A batch signature's graph, with the layout (and the descriptors uploaded for it) that
// the graph's launches read; valid while the workspace keeps its generation.
struct CachedGraph {
    cudaGraphExec_t exec = nullptr;
    uint64_t generation = 0;
    cudaEvent_t marks[N_MARKS] = {};
    std::shared_ptr<BatchLayout> layout;
    size_t ws_bytes = 0;
};
std::map<std::string, CachedGraph> g_graphs;
// signature whose descriptors the workspace of each device currently holds
std::map<int, std::string> g_uploaded;

int batch_ws_get(size_t bytes, void** out, uint64_t* generation) {
    int dev = 0;
    KNN_CK(cudaGetDevice(&dev));
    BatchWs& w = g_bws[dev];
    if (w.bytes < bytes) {
        if (w.ptr) {
            KNN_CK(cudaDeviceSynchronize());
            KNN_CK(cudaFree(w.ptr));
            w.ptr = nullptr;
        }
        const size_t want = bytes + bytes / 8;
        cudaError_t e = cudaMalloc(&w.ptr, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            w.ptr = nullptr;
            w.bytes = 0;
            return set_error(KNN_ENOMEM, "batch workspace of %zu bytes: %s", want, cudaGetErrorString(e));
        }
        w.bytes = want;
        ++w.generation;
    }
    *out = w.ptr;
    *generation = w.generation;
    return KNN_OK;
}

struct BatchLayout {
    std::vector<BatchDev> dev;          // host copies of the descriptors
    std::vector<FusedProblem> fprob;    // fused problems' kernel descriptors
    std::vector<int> fused_ids, plain_ids;
    std::vector<BatchSeg> prep_segs, query_segs, plain_prep_segs, plain_query_segs;
    std::vector<FusedWork> work;
    int64_t prep_rows = 0, query_rows = 0, plain_prep_rows = 0, plain_query_rows = 0;
    int cap_max = 0, stages = 0, grid = 0;
    // the fused work runs as up to three launches: problems on 128 x 256 tiles whose lists
    // hold at most 512 keys (the kernel variant with 16 keys a lane and four pipeline stages),
    // then the longer lists, then the problems on 128 x 128 tiles (two CTAs an SM)
    struct Part {
        int first = 0, count = 0, cap = 0, bn = 256;
    };
    Part parts[3];
    int sms = 0;
    // device pointers
    BatchDev* d_dev = nullptr;
    FusedProblem* d_fprob = nullptr;
    BatchSeg *d_prep_segs = nullptr, *d_query_segs = nullptr, *d_plain_prep_segs = nullptr,
             *d_plain_query_segs = nullptr;
    FusedWork* d_work = nullptr;
    RerankCounters* counters = nullptr;
    int* status = nullptr;
    uint64_t* scratch = nullptr;
    PrepGlobals* globals = nullptr;     // 2 per problem (queries, corpus), read back in one copy
    // plain problems share one set of slab buffers (they run one after another)
    float* slab = nullptr;
    uint64_t* slab_cand = nullptr;
    int32_t* slab_count = nullptr;
    uint64_t* slab_bound = nullptr;
    uint32_t* slab_flags = nullptr;
    int64_t slab_rows = 0, slab_cols = 0;
    int slab_cap = 0;
};

// Lays out every buffer of the batch in an arena (sizing pass when the arena has no base).
void layout_batch(const std::vector<Problem>& probs, const std::vector<int>& sched, int prec, int sms, Arena& ar,
                  BatchLayout& L) {
    const int n = static_cast<int>(probs.size());
    L.dev.assign(n, BatchDev{});
    L.globals = ar.take<PrepGlobals>(2 * static_cast<size_t>(std::max(n, 1)));
    L.fused_ids.clear();
    L.plain_ids.clear();
    for (int i = 0; i < n; ++i) (is_fused(sched[i]) ? L.fused_ids : L.plain_ids).push_back(i);
    L.cap_max = 0;
    int64_t plain_slab_bytes = 0;
    L.slab_rows = 0;
    L.slab_cols = 0;
    L.slab_cap = 0;
    for (int i = 0; i < n; ++i) {
        const Problem& p = probs[i];
        BatchDev& b = L.dev[i];
        const bool fused = is_fused(sched[i]);
        const int km = static_cast<int>(std::min<int64_t>(p.k + p.m, p.N - (p.graph ? 1 : 0)));
        b.Q = p.Q;
        b.C = p.C;
        b.M = p.M;
        b.N = p.N;
        b.d = p.d;
        b.k = p.k;
        b.km = km;
        b.graph = p.graph ? 1 : 0;
        b.vec = (p.d % 4 == 0) && (reinterpret_cast<uintptr_t>(p.Q) % 16 == 0) &&
                (reinterpret_cast<uintptr_t>(p.C) % 16 == 0);
        const int64_t n_pad = (p.N + 255) / 256 * 256;
        b.gq = L.globals ? L.globals + 2 * i : nullptr;
        b.gc = p.graph ? b.gq : (L.globals ? L.globals + 2 * i + 1 : nullptr);
        b.cnorm2 = ar.take<float>(n_pad);
        b.qnorm2 = p.graph ? b.cnorm2 : ar.take<float>(p.M);
        b.E = ar.take<float>(p.M);
        b.out_idx = p.out_idx;
        b.out_dist = p.out_dist;
        b.row_status = ar.take<uint32_t>(p.M);
        if (fused) {
            const int elem = prec == P_BF16 ? 2 : 1;
            const int per = 128 / elem;
            b.d_pad = (p.d + per - 1) / per * per;
            b.cap = fused_cap(p.k, km);
            L.cap_max = std::max(L.cap_max, b.cap);
            const size_t row_bytes = static_cast<size_t>(b.d_pad) * elem;
            b.cres = ar.take<float>(n_pad);
            b.ctn = ar.take<float>(n_pad);
            b.qres = p.graph ? b.cres : ar.take<float>(p.M);
            b.qtn = p.graph ? b.ctn : ar.take<float>(p.M);
            b.xc = ar.take<char>(row_bytes * p.N);
            b.xq = p.graph ? b.xc : ar.take<char>(row_bytes * p.M);
            if (prec == P_FP8) {
                b.cscale = ar.take<float>(n_pad);
                b.qscale = p.graph ? b.cscale : ar.take<float>(p.M);
            }
            b.E32 = ar.take<float>(p.M);
            b.cand = ar.take<uint64_t>(static_cast<size_t>(p.M) * b.cap);
            b.count = ar.take<int32_t>(p.M);
            b.bound = ar.take<uint64_t>(p.M);
            b.flags = ar.take<uint32_t>(p.M);
        } else {
            b.d_pad = p.d;
            b.cap = pick_cap(p.k, km);
            b.E32 = b.E;
            const int64_t ldn = (p.N + 31) / 32 * 32;
            const int64_t R = std::min<int64_t>((p.M + 127) / 128 * 128, std::max<int64_t>(128, (int64_t(1) << 30) / (ldn * 4) / 128 * 128));
            plain_slab_bytes = std::max<int64_t>(plain_slab_bytes, R * ldn * 4);
            L.slab_rows = std::max(L.slab_rows, R);
            L.slab_cols = std::max(L.slab_cols, ldn);
            L.slab_cap = std::max(L.slab_cap, b.cap);
        }
    }
    // segment tables and the work list
    L.prep_segs.clear();
    L.query_segs.clear();
    L.plain_prep_segs.clear();
    L.plain_query_segs.clear();
    L.work.clear();
    L.prep_rows = L.query_rows = L.plain_prep_rows = L.plain_query_rows = 0;
    for (int i : L.fused_ids) {
        L.prep_segs.push_back({L.prep_rows, i, 0});
        L.prep_rows += probs[i].N;
        if (!probs[i].graph) {
            L.prep_segs.push_back({L.prep_rows, i, 1});
            L.prep_rows += probs[i].M;
        }
        L.query_segs.push_back({L.query_rows, i, 1});
        L.query_rows += probs[i].M;
    }
    for (int i : L.plain_ids) {
        L.plain_prep_segs.push_back({L.plain_prep_rows, i, 0});
        L.plain_prep_rows += probs[i].N;
        if (!probs[i].graph) {
            L.plain_prep_segs.push_back({L.plain_prep_rows, i, 1});
            L.plain_prep_rows += probs[i].M;
        }
        L.plain_query_segs.push_back({L.plain_query_rows, i, 1});
        L.plain_query_rows += probs[i].M;
    }
    L.fprob.assign(L.fused_ids.size(), FusedProblem{});
    L.sms = sms;
    for (int pass = 0; pass < 3; ++pass) {
        const size_t first = L.work.size();
        BatchLayout::Part& part = L.parts[pass];
        part = BatchLayout::Part{};
        part.first = static_cast<int>(first);
        part.bn = pass == 2 ? 128 : 256;
        for (size_t f = 0; f < L.fused_ids.size(); ++f) {
            const int i = L.fused_ids[f];
            const Problem& p = probs[i];
            const int cap = L.dev[i].cap;
            const int bn = tile_of(sched[i]);
            if (bn != part.bn || (bn == 256 && (cap <= 512) != (pass == 0))) continue;
            part.cap = std::max(part.cap, cap);
            const int nrb = static_cast<int>((p.M + 127) / 128);
            for (int rb = 0; rb < nrb; ++rb) L.work.push_back({static_cast<int32_t>(f), rb});
        }
        // largest items first: cost of a row block ~ corpus tiles x k-steps
        std::stable_sort(L.work.begin() + static_cast<std::ptrdiff_t>(first), L.work.end(),
                         [&](const FusedWork& a, const FusedWork& b) {
                             const Problem& pa = probs[L.fused_ids[a.problem]];
                             const Problem& pb = probs[L.fused_ids[b.problem]];
                             return (pa.N + 255) / 256 * ((pa.d + 63) / 64) > (pb.N + 255) / 256 * ((pb.d + 63) / 64);
                         });
        part.count = static_cast<int>(L.work.size() - first);
    }
    // persistent CTAs of the widest launch (sizes the shrink scratch); stages: 0 when a part's
    // lists do not fit
    L.grid = 1;
    L.stages = L.fused_ids.empty() ? 0 : (1 << 20);
    for (const BatchLayout::Part& part : L.parts) {
        if (part.count == 0) continue;
        L.grid = std::max(L.grid, std::min(sms * (part.bn == 128 ? 2 : 1), part.count));
        L.stages = std::min(L.stages, fused_stages(part.cap, prec, false, part.bn));
    }
    L.d_dev = ar.take<BatchDev>(static_cast<size_t>(n));
    L.d_fprob = ar.take<FusedProblem>(std::max<size_t>(1, L.fprob.size()));
    L.d_prep_segs = ar.take<BatchSeg>(std::max<size_t>(1, L.prep_segs.size()));
    L.d_query_segs = ar.take<BatchSeg>(std::max<size_t>(1, L.query_segs.size()));
    L.d_plain_prep_segs = ar.take<BatchSeg>(std::max<size_t>(1, L.plain_prep_segs.size()));
    L.d_plain_query_segs = ar.take<BatchSeg>(std::max<size_t>(1, L.plain_query_segs.size()));
    L.d_work = ar.take<FusedWork>(std::max<size_t>(1, L.work.size()));
    L.counters = ar.take<RerankCounters>(1);
    L.status = ar.take<int>(1);
    L.scratch = ar.take<uint64_t>(L.cap_max > 0 ? fused_scratch_words(L.cap_max, L.grid) : 1);
    if (!L.plain_ids.empty()) {
        L.slab = ar.take<float>(static_cast<size_t>(plain_slab_bytes / 4));
        L.slab_cand = ar.take<uint64_t>(static_cast<size_t>(L.slab_rows) * L.slab_cap);
        L.slab_count = ar.take<int32_t>(L.slab_rows);
        L.slab_bound = ar.take<uint64_t>(L.slab_rows);
        L.slab_flags = ar.take<uint32_t>(L.slab_rows);
    }
}

// Every launch of the batch (graph-capturable: no host synchronisation, no allocation).
int enqueue_batch(const std::vector<Problem>& probs, int prec, const BatchLayout& L, cudaStream_t st,
                  cudaEvent_t* marks) {
    // external record nodes when captured (a plain record would only order the graph)
    auto mark = [&](int i) { return marks ? cudaEventRecordWithFlags(marks[i], st, cudaEventRecordExternal) : cudaSuccess; };
    KNN_CK(mark(0));
    KNN_CK(cudaMemsetAsync(L.counters, 0, sizeof(RerankCounters), st));
    KNN_CK(cudaMemsetAsync(L.status, 0, sizeof(int), st));
    KNN_CK(launch_batch_init(L.d_dev, static_cast<int32_t>(L.dev.size()), st));
    if (!L.fused_ids.empty()) {
        KNN_CK(launch_prep_batched(L.d_dev, L.d_prep_segs, static_cast<int32_t>(L.prep_segs.size()), L.prep_rows, prec,
                                   st));
        KNN_CK(launch_bounds_batched(L.d_dev, L.d_query_segs, static_cast<int32_t>(L.query_segs.size()), L.query_rows,
                                     prec, st));
        KNN_CK(mark(1));
        for (const BatchLayout::Part& part : L.parts) {
            if (part.count <= 0) continue;
            FusedParams fp{};
            fp.status = L.status;
            fp.scratch = L.scratch;
            fp.cap_max = part.cap;
            fp.stages = fused_stages(part.cap, prec, false, part.bn);
            fp.n_items = part.count;
            fp.problems = L.d_fprob;
            fp.work = L.d_work + part.first;
            const int ctas = L.sms * (part.bn == 128 ? 2 : 1);
            KNN_CK(launch_fused_batched(fp, prec, std::min(ctas, part.count), st, part.bn));
        }
        KNN_CK(mark(2));
        KNN_CK(launch_rerank_batched(L.d_dev, L.d_query_segs, static_cast<int32_t>(L.query_segs.size()), L.query_rows,
                                     L.cap_max, L.counters, st));
    } else {
        KNN_CK(mark(1));
        KNN_CK(mark(2));
    }
    KNN_CK(mark(3));
    if (!L.plain_ids.empty()) {
        KNN_CK(launch_prep_batched(L.d_dev, L.d_plain_prep_segs, static_cast<int32_t>(L.plain_prep_segs.size()),
                                   L.plain_prep_rows, P_FP32, st));
        KNN_CK(launch_bounds_batched(L.d_dev, L.d_plain_query_segs, static_cast<int32_t>(L.plain_query_segs.size()),
                                     L.plain_query_rows, P_FP32, st));
        for (int i : L.plain_ids) {
            const Problem& p = probs[i];
            const BatchDev& b = L.dev[i];
            const int km = static_cast<int>(std::min<int64_t>(p.k + p.m, p.N - (p.graph ? 1 : 0)));
            const int64_t ldn = (p.N + 31) / 32 * 32;
            const int64_t R = std::min<int64_t>((p.M + 127) / 128 * 128,
                                                std::max<int64_t>(128, (int64_t(1) << 30) / (ldn * 4) / 128 * 128));
            for (int64_t r0 = 0; r0 < p.M; r0 += R) {
                const int64_t rows = std::min<int64_t>(R, p.M - r0);
                KNN_CK(launch_gemm_simt(p.Q + r0 * p.d, rows, 0, p.C, p.N, p.d, b.cnorm2, nullptr, L.slab, ldn, 0, st));
                SelectParams sp{};
                sp.D = L.slab;
                sp.ldd = ldn;
                sp.M = rows;
                sp.N = p.N;
                sp.spec = select_spec(sp.N);
                sp.k = p.k;
                sp.km = km;
                sp.cap = b.cap;
                sp.E = b.E + r0;
                sp.cand = L.slab_cand;
                sp.count = L.slab_count;
                sp.bound = L.slab_bound;
                sp.flags = L.slab_flags;
                KNN_CK(launch_select_ex(sp, p.graph ? r0 : -1, false, st));
                RerankParams rp{};
                rp.Q = p.Q + r0 * p.d;
                rp.C = p.C;
                rp.M = rows;
                rp.N = p.N;
                rp.d = p.d;
                rp.k = p.k;
                rp.km = km;
                rp.cap = b.cap;
                rp.cand = L.slab_cand;
                rp.count = L.slab_count;
                rp.bound = L.slab_bound;
                rp.flags = L.slab_flags;
                rp.E = b.E + r0;
                rp.out_idx = p.out_idx + r0 * p.k;
                rp.out_dist = p.out_dist + r0 * p.k;
                rp.row_status = b.row_status + r0;
                rp.counters = L.counters;
                rp.uncertified = &b.gq->uncertified;
                KNN_CK(launch_rerank(rp, st));
            }
        }
    }
    KNN_CK(mark(4));
    return KNN_OK;
}

std::string signature(const std::vector<Problem>& probs, const std::vector<int>& sched, int prec) {
    std::string s;
    char b[160];
    std::snprintf(b, sizeof(b), "p%d|", prec);
    s += b;
    for (size_t i = 0; i < probs.size(); ++i) {
        const Problem& p = probs[i];
        std::snprintf(b, sizeof(b), "%p,%p,%lld,%lld,%d,%d,%d,%d,%d,%p,%p;", (const void*)p.Q, (const void*)p.C,
                      (long long)p.M, (long long)p.N, p.d, p.k, p.m, p.graph ? 1 : 0, sched[i], (void*)p.out_idx,
                      (void*)p.out_dist);
        s += b;
    }
    return s;
}


// Forgets a batch's cached graph (the autotuner's one-problem timing batches, whose buffers are
// freed right after).
void drop_batch_graph(const std::vector<Problem>& probs, const std::vector<int>& sched, int prec) {
    const std::string sig = signature(probs, sched, prec);
    std::lock_guard<std::mutex> lk(g_bws_mu);
    auto it = g_graphs.find(sig);
    if (it == g_graphs.end()) return;
    if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
    for (auto e : it->second.marks)
        if (e) cudaEventDestroy(e);
    g_graphs.erase(it);
    for (auto& kv : g_uploaded)
        if (kv.second == sig) kv.second.clear();
}

}  // namespace

// Runs the batch (device pointers only); per-problem statuses in status[]. Returns the
// first failure or KNN_OK.
int run_batch(std::vector<Problem>& probs, std::vector<int>& status, int precision_req, ::knn_stats* stats,
              cudaStream_t st) {
    const auto t_call = std::chrono::steady_clock::now();
    const int n = static_cast<int>(probs.size());
    std::vector<int> sched(n, SCHED_PLAIN);
    int prec = precision_req == KNN_FP8_E4M3 ? P_FP8 : P_BF16;
    for (int i = 0; i < n; ++i) {
        bool capable = false;
        sched[i] = choose_schedule(probs[i], precision_req, &capable);
    }
    int dev = 0, sms = 0;
    KNN_CK(cudaGetDevice(&dev));
    KNN_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // the graph, layout and descriptors are kept per batch signature; a repeated call with
    // the same signature and workspace only launches the graph
    const std::string sig = signature(probs, sched, prec);
    std::lock_guard<std::mutex> lk(g_bws_mu);
    CachedGraph& cg = g_graphs[sig];
    void* base = nullptr;
    uint64_t gen = 0;
    std::shared_ptr<BatchLayout> Lp;
    if (cg.exec && cg.layout) {
        KNN_TRY(batch_ws_get(cg.ws_bytes, &base, &gen));
        if (gen == cg.generation) Lp = cg.layout;
    }
    if (!Lp) {
        Lp = std::make_shared<BatchLayout>();
        BatchLayout& L = *Lp;
        Arena sz;
        layout_batch(probs, sched, prec, sms, sz, L);
        if (!L.fused_ids.empty() && L.stages == 0) {
            for (int i : L.fused_ids) sched[i] = SCHED_PLAIN;  // cannot happen: capable problems fit
            Arena sz2;
            L = BatchLayout{};
            layout_batch(probs, sched, prec, sms, sz2, L);
            sz = sz2;
        }
        KNN_TRY(batch_ws_get(sz.used(), &base, &gen));
        Arena ar(static_cast<char*>(base), sz.used());
        L = BatchLayout{};
        layout_batch(probs, sched, prec, sms, ar, L);
        // descriptors: tensor maps of the fused problems
        for (size_t f = 0; f < L.fused_ids.size(); ++f) {
            const int i = L.fused_ids[f];
            const BatchDev& b = L.dev[i];
            FusedProblem& q = L.fprob[f];
            const int km =
                static_cast<int>(std::min<int64_t>(probs[i].k + probs[i].m, probs[i].N - (probs[i].graph ? 1 : 0)));
            q.M = b.M;
            q.N = b.N;
            q.k_bytes = b.d_pad * (prec == P_BF16 ? 2 : 1);
            q.k = b.k;
            q.km = km;
            q.cap = b.cap;
            q.self_offset = b.graph ? 0 : -1;
            q.cnorm2 = b.cnorm2;
            q.E = b.E;
            q.thr = nullptr;
            q.q_inv_scale = b.qscale;
            q.c_inv_scale = b.cscale;
            q.cand = b.cand;
            q.count = b.count;
            q.bound = b.bound;
            q.flags = b.flags;
            // speculation as the autotuner chose it, else from 16384 points on
            const int sc = sched[L.fused_ids[f]];
            q.spec = spec_of(sc) >= 0 ? spec_of(sc) : (b.N >= 16384 ? 1 : 0);
            if (!encode_problem_maps(&q, b.xq, b.xc, prec, tile_of(sc)))
                return set_error(KNN_EUNSUPPORTED, "tensor map encoding failed for problem %d", i);
        }
        if (cg.exec) {
            cudaGraphExecDestroy(cg.exec);  // captured for another workspace
            cg.exec = nullptr;
        }
        cg.layout = nullptr;
        cg.ws_bytes = sz.used();
        g_uploaded[dev].clear();
    }
    BatchLayout& L = *Lp;
    if (g_uploaded[dev] != sig) {
        // the descriptors to the device (the layout's host vectors outlive the copies)
        KNN_CK(cudaMemcpyAsync(L.d_dev, L.dev.data(), L.dev.size() * sizeof(BatchDev), cudaMemcpyHostToDevice, st));
        if (!L.fprob.empty())
            KNN_CK(cudaMemcpyAsync(L.d_fprob, L.fprob.data(), L.fprob.size() * sizeof(FusedProblem),
                                   cudaMemcpyHostToDevice, st));
        auto put = [&](auto* dst, const auto& v) -> cudaError_t {
            if (v.empty()) return cudaSuccess;
            return cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice, st);
        };
        KNN_CK(put(L.d_prep_segs, L.prep_segs));
        KNN_CK(put(L.d_query_segs, L.query_segs));
        KNN_CK(put(L.d_plain_prep_segs, L.plain_prep_segs));
        KNN_CK(put(L.d_plain_query_segs, L.plain_query_segs));
        KNN_CK(put(L.d_work, L.work));
        g_uploaded[dev] = sig;
    }

    // the graph: captured once per batch signature, replayed afterwards
    if (!cg.marks[0])
        for (auto& e : cg.marks) KNN_CK(cudaEventCreate(&e));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!cg.exec) {
        cudaStream_t cs = nullptr;
        KNN_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        KNN_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue_batch(probs, prec, L, cs, cg.marks);
        const cudaError_t ec = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (rc != KNN_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        KNN_CK(ec);
        const cudaError_t ei = cudaGraphInstantiate(&cg.exec, g, 0);
        cudaGraphDestroy(g);
        KNN_CK(ei);
        cg.generation = gen;
        cg.layout = Lp;
    }
    KNN_CK(cudaEventCreate(&e0));
    KNN_CK(cudaEventCreate(&e1));
    KNN_CK(cudaEventRecord(e0, st));
    KNN_CK(cudaGraphLaunch(cg.exec, st));
    KNN_CK(cudaEventRecord(e1, st));
    RerankCounters hc{};
    int hstatus = 0;
    std::vector<PrepGlobals> hg(2 * static_cast<size_t>(n));
    KNN_CK(cudaMemcpyAsync(&hc, L.counters, sizeof(hc), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaMemcpyAsync(&hstatus, L.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaMemcpyAsync(hg.data(), L.globals, hg.size() * sizeof(PrepGlobals), cudaMemcpyDeviceToHost, st));
    KNN_CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    float phase[N_MARKS - 1] = {};
    for (int i = 0; i + 1 < N_MARKS; ++i)
        if (cudaEventElapsedTime(&phase[i], cg.marks[i], cg.marks[i + 1]) != cudaSuccess) {
            cudaGetLastError();
            phase[i] = -1.f;
        }
    if (hstatus != 0) return set_error(KNN_ETIMEOUT, "the batched fused kernel stopped: a device-side wait timed out");

    // per problem: NaN/Inf inputs, then rows the batch could not certify
    int first = KNN_OK;
    int64_t fallback_rows = 0;
    for (int i = 0; i < n; ++i) {
        const PrepGlobals& gq = hg[2 * static_cast<size_t>(i)];
        const PrepGlobals& gc = probs[i].graph ? gq : hg[2 * static_cast<size_t>(i) + 1];
        if (gq.nonfinite || gc.nonfinite) {
            status[i] = set_error(KNN_EINVAL, "problem %d: input holds NaN or Inf", i);
            if (first == KNN_OK) first = status[i];
        }
    }
    if (hc.uncertified > 0) {
        std::vector<uint32_t> rs;
        for (int i = 0; i < n; ++i) {
            // the re-rank counted each problem's uncertified rows in its query statistics
            if (status[i] != KNN_OK || hg[2 * static_cast<size_t>(i)].uncertified == 0) continue;
            const BatchDev& b = L.dev[i];
            rs.resize(static_cast<size_t>(b.M));
            KNN_CK(cudaMemcpyAsync(rs.data(), b.row_status, b.M * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            KNN_CK(cudaStreamSynchronize(st));
            std::vector<int32_t> bad;
            for (int64_t r = 0; r < b.M; ++r)
                if (rs[static_cast<size_t>(r)] & ROW_UNCERTIFIED) bad.push_back(static_cast<int32_t>(r));
            if (bad.empty()) continue;
            // rare: recompute those rows exactly (plain FP32 form, then FP64)
            Problem q = probs[i];
            q.precision = KNN_FP32;
            q.fused = 0;
            const int rc = recompute_rows(q, bad, st);
            fallback_rows += static_cast<int64_t>(bad.size());
            if (rc != KNN_OK) {
                status[i] = rc;
                if (first == KNN_OK) first = rc;
            }
        }
    }
    if (stats) {
        int64_t rows = 0;
        for (const Problem& p : probs) rows += p.M;
        stats->rows = rows;
        stats->candidates = static_cast<int64_t>(hc.candidates);
        stats->rows_truncated = static_cast<int64_t>(hc.truncated);
        stats->rows_uncertified = static_cast<int64_t>(hc.uncertified);
        stats->rows_fallback = fallback_rows;
        stats->rows_fp64_ties = static_cast<int64_t>(hc.fp64_rows);
        {
            const uint32_t bits = static_cast<uint32_t>(hc.max_err_ratio);
            std::memcpy(&stats->max_error_ratio, &bits, sizeof(float));
        }
        // device phases of the graph; ms_total is the whole call on the host, so
        // ms_total - ms_gemm is the host work around the graph
        stats->ms_total = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t_call).count();
        stats->ms_gemm = ms;
        stats->ms_prep = phase[0];
        stats->ms_select = phase[1];
        stats->ms_rerank = phase[2];
        stats->ms_fallback = phase[3];
        stats->fused_used = static_cast<int32_t>(L.fused_ids.size());
        stats->list_capacity = L.cap_max;
        stats->precision_used = prec == P_BF16 ? KNN_BF16 : KNN_FP8_E4M3;
        stats->gemm_launches = 1;
        double flops = 0.0;
        for (const Problem& p : probs) flops += 2.0 * double(p.M) * double(p.N) * double(p.d);
        stats->gemm_flops = flops;
        stats->kernel_launches =
            1 + (L.fused_ids.empty() ? 0 : 2 + (L.parts[0].count > 0) + (L.parts[1].count > 0) + (L.parts[2].count > 0) +
                                                rerank_launches(L.cap_max)) +
            (L.plain_ids.empty() ? 0 : 2);
        for (int i : L.plain_ids) {
            const Problem& p = probs[i];
            const int64_t ldn = (p.N + 31) / 32 * 32;
            const int64_t R = std::min<int64_t>((p.M + 127) / 128 * 128,
                                                std::max<int64_t>(128, (int64_t(1) << 30) / (ldn * 4) / 128 * 128));
            const int km = static_cast<int>(std::min<int64_t>(p.k + p.m, p.N - (p.graph ? 1 : 0)));
            stats->kernel_launches += (2 + rerank_launches(pick_cap(p.k, km))) * ((p.M + R - 1) / R);
        }
    }
    return first;
}

}  // namespace knn
