// Host-side declarations shared by the engine's translation units (not part of the ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace knn {

enum Precision : int32_t { P_FP32 = 0, P_BF16 = 1, P_FP8 = 2 };

// Statistics of one point set gathered by the prep kernel (device memory, zeroed before use).
// Non-negative floats are stored as their bit patterns, whose unsigned order is the value order.
struct PrepGlobals {
    uint32_t max_norm2;   // max |x|^2
    uint32_t max_abs;     // max |x_t|
    uint32_t max_res;     // max |x - x~| (x~ = reduced-precision copy)
    uint32_t max_tnorm;   // max |x~|
    uint32_t nonfinite;   // rows holding NaN or Inf
    uint32_t noninteger;  // rows holding a non-integer value
    uint32_t uncertified; // query rows the re-rank left uncertified (batched form, query side)
    uint32_t pad;
};

// Per-row candidate state handed from the select to the re-rank.
enum RowFlag : uint32_t {
    ROW_TRUNCATED = 1u,       // candidate list reached capacity; the bound decides exactness
    ROW_THRESHOLD_MISS = 2u,  // a supplied threshold kept fewer than k candidates
    ROW_SELECT_ERROR = 4u,    // the select gave up (iteration limit)
    ROW_SPECULATIVE = 8u,     // a speculative threshold was used: the band must be checked against the bound
    ROW_RAW_LIST = 16u,       // the list holds every key <= bound, not yet reduced to the band, in two
                              // segments: count = front | back << 16, the back filled from cand[cap - 1] down
    ROW_BOUNDED = 32u,        // a bounding threshold (Problem::thr_bound) was supplied and the list holds
                              // every key at or below it: exact among the points within the bound
};

enum RowStatus : uint32_t {
    ROW_UNCERTIFIED = 1u,  // the re-rank could not prove the answer exact
    ROW_FP64 = 2u,         // FP64 decided a near tie in this row
    ROW_RERANKED = 4u,     // the re-rank has written this row's answer
};

// Counters accumulated by the re-rank (device memory, zeroed per call).
struct RerankCounters {
    unsigned long long candidates;
    unsigned long long fp64_rows;
    unsigned long long uncertified;
    unsigned long long truncated;
    unsigned long long threshold_miss;
    unsigned long long inserted;  // keys the fused sweep appended to candidate lists
    unsigned long long max_err_ratio;  // float bits of the largest |approximate - exact| / E of a candidate
    unsigned long long rows_in_sweep;  // rows re-ranked by the fused kernel during its sweep
    unsigned long long next_row[4];    // work counters of the re-rank launches (one per list-length tier)
};

// ---- prep / bounds (prep.cu) ----
// Raises a kernel's dynamic shared-memory limit on the current device to at least `bytes`
// and never lowers it: a kernel launched with several sizes (re-rank tiers, list
// capacities) keeps every launch recorded earlier valid, including kernel nodes of a
// captured graph that are launched again on their own (as a profiler's replay does).
cudaError_t raise_smem_limit(const void* kernel, size_t bytes);

cudaError_t launch_prep(const float* X, int64_t rows, int32_t d, int32_t precision, float* norm2, float* res,
                        float* tnorm, void* xq, int32_t ldq, float* inv_scale, PrepGlobals* g, cudaStream_t st);

// E[i]: bound on |approximate - exact| of every d'_ij of row i (0 in exact arithmetic).
// With sym_extra, E also covers the two extra roundings of the symmetric form's transposed keys.
cudaError_t launch_bounds(const float* qnorm2, const float* qres, const float* qtnorm, int64_t M, int32_t d,
                          int32_t d_pad, int32_t precision, const PrepGlobals* gq, const PrepGlobals* gc, float* E,
                          cudaStream_t st, bool sym_extra = false);

// ---- FP32 SIMT distance GEMM (gemm_simt.cu) ----
// D[i*ldd + j] = cnorm2[j] - 2 q_i.c_j (+ qnorm2[i] when qnorm2 != nullptr); +inf where
// exclude_self and row0 + i == j.
cudaError_t launch_gemm_simt(const float* Q, int64_t M, int64_t row0, const float* C, int64_t N, int32_t d,
                             const float* cnorm2, const float* qnorm2, float* D, int64_t ldd, int32_t exclude_self,
                             cudaStream_t st);

// ---- quick multi-select (select.cu) ----
struct SelectParams {
    const float* D;        // M x N values, row stride ldd
    int64_t ldd, M, N;
    int32_t k, km;         // answer size and always-kept candidate count (km >= k)
    int32_t cap;           // candidate list capacity per row (>= km)
    const float* E;        // per-row error bound (window = 2E); nullptr = 0
    const float* thr;      // per-row initial threshold in D's scale; nullptr = none
    uint64_t* cand;        // M x cap keys (value, column)
    int32_t* count;        // M
    uint64_t* bound;       // M: every key left out of the list is > bound[i]
    uint32_t* flags;       // M: RowFlag bits
    const int32_t* self_col;  // per-row excluded column (or nullptr)
    int32_t spec;          // 1: speculative thresholds while streaming a row (rows they fail are redone)
    int32_t block;         // 1: one CTA per row (sorted select only; see select_prefers_block)
};
cudaError_t launch_select(const SelectParams& p, cudaStream_t st);
// Whether rows of length N are selected with speculative thresholds (SelectParams::spec):
// from 16384 columns on; KNN_SPECULATE=0/1 overrides.
int select_spec(int64_t N);
// Segments per row for a select of few long dense rows (1: no split): each row of length N is
// selected as S rows of N / S columns, then merged by launch_select_merge.
int select_split_segments(int64_t M, int64_t N, int64_t ldd, int32_t k, const void* D);
// Row r's answer from its S segment answers (rows r S .. r S + S - 1 of seg_idx/seg_val, k
// each, segment-local indices); flags[r] = OR of the segments' flags.
cudaError_t launch_select_merge(const int32_t* seg_idx, const float* seg_val, const uint32_t* seg_flags, int64_t M,
                                int32_t S, int32_t k, int64_t seg_len, int32_t* out_idx, float* out_val,
                                uint32_t* flags, cudaStream_t st);

// Row r's indices from a select over the concatenation of its S segment answers (M x S k
// values): merged_col[r][i] is a column of that concatenation; out_idx[r][i] the row's global
// column; flags[r] |= OR of the segments' flags.
cudaError_t launch_select_remap(const int32_t* merged_col, const int32_t* seg_idx, const uint32_t* seg_flags,
                                int64_t M, int32_t S, int32_t k, int64_t seg_len, int32_t* out_idx, uint32_t* flags,
                                cudaStream_t st);

// Smallest k whose sorted select runs one CTA per row instead of one warp (128;
// KNN_SELECT_BLOCK_K overrides: 0 = never, 1 = always).
int select_block_k();
// Whether a sorted select of M rows takes one CTA per row: for k >= select_block_k(), and
// for at most 64 rows (one warp per row leaves the GPU idle there, even after a split).
bool select_prefers_block(int64_t M, int32_t k);

// Select output written directly as sorted (index, value) pairs: the k smallest per row.
cudaError_t launch_select_topk(const SelectParams& p, int32_t* out_idx, float* out_val, cudaStream_t st);

// ---- exact re-rank (rerank.cu) ----
struct RerankParams {
    const float* Q;        // M x d queries (rows of this slab)
    const float* C;        // N x d corpus
    int64_t M, N;
    int32_t d, k, km, cap;  // km: keys the band keeps at least (k + m)
    const uint64_t* cand;  // M x cap
    const int32_t* count;
    const uint64_t* bound;
    const uint32_t* flags;
    const float* E;        // per-row bound used for the candidates' approximate values
    int32_t* out_idx;      // M x k
    float* out_dist;       // M x k
    uint32_t* row_status;  // M
    RerankCounters* counters;
    int32_t count_min, count_max;  // rows whose list length lies outside are skipped (set by launch_rerank)
    int32_t skip_done;     // 1: rows whose row_status has ROW_RERANKED are skipped (re-ranked earlier)
    const int* status;     // optional device status word: when non-zero nothing is re-ranked
    // symmetric graph form: keys of the transposed pairs of row i in inbox[i * cap_in ...],
    // inbox_cnt[i] of them (more than cap_in: keys were lost and the row is not certified)
    const uint64_t* inbox;
    const int32_t* inbox_cnt;
    int32_t cap_in;
    uint32_t* uncertified;  // optional: counts the rows left uncertified (one atomic per such row)
};
// Lists longer than 512 (and 1024) keys are re-ranked by further launches with larger
// per-warp buffers, so the common short lists keep the higher occupancy.
cudaError_t launch_rerank(const RerankParams& p, cudaStream_t st);
inline int rerank_launches(int keys) { return keys > 1024 ? 3 : (keys > 512 ? 2 : 1); }

// ---- band probe (probe.cu) ----
// out_count[i] = #{ j != self_col[i] : D[i][j] <= max(vals[i][km-1], vals[i][k-1] + 2 E[i]) },
// vals[i] holding row i's km smallest values in ascending order; out_count4[i] (optional) the
// same with 4 E (the reach of a band taken on approximate values); out_edge[i] (optional) =
// the 2 E band edge plus qnorm2[row_ids[i]], a squared distance.
cudaError_t launch_band_count(const float* D, int64_t rows, int64_t N, int64_t ldd, const float* vals, int32_t k,
                              int32_t km, const float* E, const int32_t* self_col, const float* qnorm2,
                              const int32_t* row_ids, int32_t* out_count, int32_t* out_count4, float* out_edge,
                              cudaStream_t st);

// out[i] = #{ j != self_col[i] : D[i][j] + qnorm2[row_ids[i]] <= t } for the sampled rows: the
// keys at or below the squared distance t (the most the symmetric form sends to a row's inbox).
cudaError_t launch_count_le(const float* D, int64_t rows, int64_t N, int64_t ldd, float t, const float* qnorm2,
                            const int32_t* row_ids, const int32_t* self_col, int32_t* out, cudaStream_t st);

// ---- batched problems (batched.cu, with batched kernels in prep.cu / rerank.cu) ----
// Device-side description of one problem of a batch and of its buffers.
struct BatchDev {
    const float* Q;           // M x d queries (== C for a graph)
    const float* C;           // N x d corpus
    int64_t M, N;
    int32_t d, k, km, cap, d_pad;
    int32_t graph;            // 1: k-NN graph (self excluded, one prep)
    int32_t vec;              // 1: 16-byte aligned rows (d % 4 == 0)
    PrepGlobals* gq;
    PrepGlobals* gc;
    float *qnorm2, *cnorm2, *qres, *cres, *qtn, *ctn, *qscale, *cscale;
    void* xq;
    void* xc;
    float* E;                 // bound of the reduced-precision form
    float* E32;               // bound of the FP32 form (fallback)
    uint64_t* cand;
    int32_t* count;
    uint64_t* bound;
    uint32_t* flags;
    int32_t* out_idx;
    float* out_dist;
    uint32_t* row_status;
};

// A run of consecutive global rows that belong to one matrix of one problem.
struct BatchSeg {
    int64_t row0;     // first global row of the segment
    int32_t problem;
    int32_t which;    // 0: corpus rows, 1: query rows
};

// Per-problem initialisation of a batch in one launch: the prep statistics zeroed, and
// the corpus norms of the tensor-core problems (those with a reduced-precision copy)
// padded past N to a multiple of 256 with NaN, so that padded columns never pass.
cudaError_t launch_batch_init(const BatchDev* probs, int32_t n, cudaStream_t st);
// Prep of every corpus (and non-graph query) row of the batch; segs sorted by row0.
cudaError_t launch_prep_batched(const BatchDev* probs, const BatchSeg* segs, int32_t nseg, int64_t rows,
                                int32_t precision, cudaStream_t st);
// Bounds (reduced-precision E and FP32 E32) of every query row; segs over query rows.
cudaError_t launch_bounds_batched(const BatchDev* probs, const BatchSeg* segs, int32_t nseg, int64_t rows,
                                  int32_t precision, cudaStream_t st);
// Exact re-rank of every query row; cap_max sizes the shared memory.
cudaError_t launch_rerank_batched(const BatchDev* probs, const BatchSeg* segs, int32_t nseg, int64_t rows,
                                  int32_t cap_max, RerankCounters* counters, cudaStream_t st);

// ---- cosine and Pearson similarity (metric.cu) ----
// Per row: FP64 mean (centered) and norm of the centred row, and the FP32 unit row
// (x - mean) / norm; *bad |= 1 for a zero, NaN or infinite norm.
cudaError_t launch_sim_prep(const float* X, int64_t rows, int32_t d, int32_t centered, float* U, double* mean,
                            double* norm, int32_t* bad, cudaStream_t st);
struct SimRerankParams {
    const float* Q;            // M x d original queries
    const float* C;            // N x d original corpus
    const double* qmean;
    const double* qnorm;
    const double* cmean;
    const double* cnorm;
    const int32_t* cand_idx;   // M x kp, nearest unit rows first
    const float* cand_dist;    // M x kp, their squared distances in the unit rows
    int64_t M;
    int32_t d, k, kp, P;       // P = power of two >= kp
    int32_t all_candidates;    // 1: the candidates are every point (nothing to certify)
    double margin;             // sim_margin(d)
    int32_t* out_idx;          // M x k
    float* out_val;            // M x k similarities
    uint32_t* uncertified;     // M
};
// Distance margin of the similarity certificate for dimension d.
double sim_margin(int32_t d);
cudaError_t launch_sim_rerank(const SimRerankParams& p, int32_t centered, cudaStream_t st);

// ---- out-of-core corpus (stream.cu) ----
struct StreamMergeParams {
    const float* Q;            // M x d queries
    const float* chunk;        // the resident chunk: rows chunk_row0 .. of the corpus
    int64_t chunk_row0;
    const int32_t* chunk_idx;  // M x kc chunk-local indices (the chunk's answer)
    int64_t M;
    int32_t d, k, kc, P;       // P = power of two >= k + kc
    int32_t* run_idx;          // M x k running answer (global indices, -1 = empty)
    double* run_d64;           // M x k their FP64 direct-difference distances
    float* run_f32;            // M x k the FP32 rounding of run_d64 (the reported distances)
};
cudaError_t launch_stream_init(int64_t n, int32_t* idx, double* d64, float* f32, cudaStream_t st);
cudaError_t launch_stream_merge(const StreamMergeParams& p, cudaStream_t st);
// thr[i] = the running k-th FP64 distance of query i rounded up to FP32 (+inf while fewer than k
// points have been merged): the bound for the next chunk's search.
cudaError_t launch_stream_bound(const double* run_d64, int64_t M, int32_t k, float* thr, cudaStream_t st);

// Exact FP64 answer for a list of rows (last-resort path; slow, used for rows no other path certifies).
cudaError_t launch_exact_rows_fp64(const float* Q, const float* C, int64_t N, int32_t d, int32_t k,
                                   int32_t exclude_self, const int32_t* rows, int32_t nrows, double* scratch,
                                   int32_t* out_idx, float* out_dist, cudaStream_t st);
// The same for cosine (centered = 0) or Pearson (centered = 1) similarity, the k most similar
// (descending, ties to the lower index), with the means and norms of launch_sim_prep.
cudaError_t launch_exact_rows_sim_fp64(const float* Q, const float* C, int64_t N, int32_t d, int32_t k,
                                       int32_t exclude_self, int32_t centered, const double* qmean,
                                       const double* qnorm, const double* cmean, const double* cnorm,
                                       const int32_t* rows, int32_t nrows, double* scratch, int32_t* out_idx,
                                       float* out_val, cudaStream_t st);

}  // namespace knn
