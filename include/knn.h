/*
 * knn.h -- C ABI of the GB300 exact brute-force k-NN / k-NN graph engine.
 *
 * The method is Komarov, Dashti and D'Souza, "Fast k-NNG construction with
 * GPU-based quick multi-select":
 *   - the k-NN problem and the k-NN graph (Introduction): for every query point,
 *     the k nearest corpus points; in the graph the corpus is the query set and a
 *     point is never its own neighbour;
 *   - distances as a matrix product (Methods, "Distance calculation"): squared
 *     Euclidean d2_ij = |x_i|^2 + |y_j|^2 - 2 x_i.y_j, ranked by the per-row
 *     equivalent d'_ij = |y_j|^2 - 2 x_i.y_j;
 *   - per-row selection of the k smallest entries by quick multi-select with warp
 *     ballot/popc partitions (Methods, "GPU-based quick multi-select").
 *
 * Results are EXACT: every row is sorted ascending by (squared distance, corpus
 * index), self excluded in the graph (by index, not by distance: duplicates still
 * appear at distance 0), ties at equal distance resolved to the lower index.
 * Reduced-precision forms (BF16, FP8) select a candidate superset that provably
 * contains the exact answer and re-rank it with direct-difference FP32 arithmetic;
 * FP64 settles near ties. Reported distances are squared and within 1e-5 relative
 * of the FP64 value (bit-exact where the inputs make FP32 arithmetic exact).
 *
 * Conventions for every entry point:
 *   - Arrays are dense, row-major and contiguous unless a leading dimension is given.
 *   - Arrays may live in device memory or in host memory; host arrays (pinned or
 *     pageable) are copied to the device and back on the call's stream.
 *   - The caller owns all inputs and outputs. The library owns its workspace, cached
 *     per device and released by knn_shutdown().
 *   - Calls are synchronous: they return once outputs are written (or on error). Calls on
 *     the same device from several host threads must be serialised by the caller: they share
 *     the device's cached workspace and staging buffers.
 *   - Errors are returned as a knn_status, never by aborting. On a non-OK status the
 *     outputs are undefined; knn_last_error() gives a message (per thread).
 *   - Indices are int32; N must be below 2^31.
 */
#ifndef KNN_H
#define KNN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum knn_status {
    KNN_OK = 0,
    KNN_EINVAL = -1,     /* bad argument: NULL pointer, k < 1, k > available points, d < 1, NaN/Inf input */
    KNN_ENOMEM = -2,     /* workspace allocation failed */
    KNN_ECUDA = -3,      /* a CUDA call failed (message in knn_last_error) */
    KNN_ETIMEOUT = -4,   /* a bounded device-side wait gave up */
    KNN_EINTERNAL = -5,  /* an internal consistency check failed */
    KNN_EUNSUPPORTED = -6 /* the requested form is not available on this device or build */
} knn_status;

typedef enum knn_precision {
    KNN_FP32 = 0,      /* SIMT FP32 distance GEMM, materialised matrix, unfused select */
    KNN_BF16 = 1,      /* tcgen05 BF16 GEMM with FP32 accumulation */
    KNN_FP8_E4M3 = 2,  /* tcgen05 FP8 e4m3 GEMM with per-row power-of-two scales */
    KNN_AUTO = -1
} knn_precision;

enum {
    KNN_FLAG_TIMING = 1 << 0,       /* fill the ms_* fields of knn_stats (CUDA events on the stream) */
    KNN_FLAG_NO_FALLBACK = 1 << 1,  /* report uncertified rows instead of recomputing them (tests) */
    KNN_FLAG_CHECK_FINITE = 1 << 2  /* reject NaN/Inf inputs with KNN_EINVAL (on by default via knn_options_init) */
};

/* Per-call statistics (optional output). */
typedef struct knn_stats {
    int64_t rows;              /* query rows answered */
    int64_t candidates;        /* candidates re-ranked exactly, summed over rows */
    int64_t rows_truncated;    /* rows whose candidate list reached its capacity */
    int64_t rows_uncertified;  /* rows the first pass could not prove exact */
    int64_t rows_fallback;     /* rows recomputed by a more precise path */
    int64_t rows_fp64_ties;    /* rows where FP64 decided a near tie */
    int64_t threshold_misses;  /* rows where a supplied threshold kept fewer than k candidates */
    float max_error_bound;     /* largest per-row bound on |approximate - exact| squared distance */
    float ms_total, ms_prep, ms_select, ms_rerank, ms_fallback; /* with KNN_FLAG_TIMING; in the plain
                                  form ms_select and ms_rerank are the device times of the select and
                                  re-rank launches alone (the slabs interleave them with the GEMM) */
    float ms_gemm;             /* with KNN_FLAG_TIMING: device time of the distance kernel (fused: GEMM + select) */
    int32_t gemm_launches;     /* launches of that kernel */
    int64_t kernel_launches;   /* every kernel the call launched */
    double gemm_flops;         /* 2 M N d_effective: the distance product the GEMM launches computed */
    int32_t precision_used;    /* knn_precision actually run */
    int32_t fused_used;        /* 1 when the select ran inside the GEMM epilogue */
    int32_t exact_arithmetic;  /* 1 when the inputs made the GEMM exact (integer-valued, small) */
    int32_t list_capacity;     /* candidate-list capacity per row of the first pass (largest in a batch) */
    int64_t candidates_inserted; /* fused form: keys the running thresholds let into candidate lists
                                    during the sweep (the select's work), summed over rows */
    float max_error_ratio;     /* largest |approximate - exact| / E_i over the candidates the re-rank
                                  evaluated, where E_i is the row's proven error bound of the GEMM's
                                  ranking value (exactness rests on this ratio staying <= 1) */
    int64_t rows_reranked_in_sweep; /* fused form: rows re-ranked by the fused kernel while it swept
                                       later row blocks (the rest by the re-rank launch after it) */
    int32_t symmetric;         /* k-NN graph: 1 when the fused launch computed each pair's product once,
                                  for both of its rows (the symmetric half of the distance product) */
} knn_stats;

typedef struct knn_options {
    int32_t precision;          /* knn_precision; KNN_AUTO picks BF16 fused where available */
    int32_t rerank_extra;       /* m: candidates beyond k always re-ranked exactly (>= 0; default 32) */
    int32_t fused;              /* -1 auto, 0 materialise the distance matrix, 1 fuse the select into the GEMM */
    int32_t flags;              /* KNN_FLAG_* */
    void* stream;               /* cudaStream_t to run on; NULL = the legacy default stream */
    const float* row_threshold; /* optional, M floats (device or host): per-row squared-distance
                                   threshold proposal that pre-filters candidates; rows where fewer
                                   than k candidates pass are recomputed without it */
    knn_stats* stats;           /* optional output */
    int64_t max_workspace_bytes;/* 0 = no cap; otherwise the call's device workspace is kept within it
                                   (distance-matrix slabs and FP64 scratch shrink to fit), and a call
                                   whose workspace cannot fit returns KNN_ENOMEM */
} knn_options;

/* Fill *opt with defaults: KNN_AUTO, m = 32, fused auto, finite check on. */
void knn_options_init(knn_options* opt);

/*
 * k-NN graph of N points X (N x d FP32). out_idx, out_dist: N x k.
 * Requires 1 <= k <= N - 1, d >= 1. (Introduction: k-NNG; Methods: distance
 * calculation and quick multi-select.) Default options.
 */
int knng_build(const float* X, int64_t N, int32_t d, int32_t k, int32_t* out_idx, float* out_dist);

/* knng_build with options (opt may be NULL for defaults). */
int knng_build_ex(const float* X, int64_t N, int32_t d, int32_t k, int32_t* out_idx, float* out_dist,
                  const knn_options* opt);

/*
 * k-NN search: for each of the M queries Q (M x d) the k nearest of the N corpus
 * points C (N x d); nothing is excluded. Requires 1 <= k <= N.
 * out_idx, out_dist: M x k.
 */
int knn_search(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k,
               int32_t* out_idx, float* out_dist, const knn_options* opt);

/* Metrics of the paper (Methods, "Distance calculation"). */
typedef enum knn_metric {
    KNN_METRIC_EUCLIDEAN = 0, /* squared Euclidean distance, ascending */
    KNN_METRIC_COSINE = 1,    /* cosine similarity x.y / (|x| |y|), descending */
    KNN_METRIC_PEARSON = 2    /* Pearson similarity: the cosine of rows centred on their own mean */
} knn_metric;

/*
 * k-NN search by a metric of the paper: for KNN_METRIC_EUCLIDEAN exactly knn_search
 * (out_val = squared distances, ascending). For KNN_METRIC_COSINE and
 * KNN_METRIC_PEARSON, out_val holds the similarities (FP32 rounding of a value within
 * 2^-38 of the FP64 similarity), each row descending by similarity, ties to the lower
 * index; the answer is exact: the nearest unit rows found by the engine are re-ranked by
 * their similarity, its dot product summed from FP32 error-free transformations in FP64
 * (within 2^-38 of sum |x_t y_t|), under a certificate that covers that error, and rows
 * it does not cover are recomputed over the whole corpus in FP64. A row of zero norm (Pearson: zero norm after
 * centring) or with a non-finite value returns KNN_EINVAL. opt->row_threshold must be
 * NULL for the similarity metrics. opt->stats: rows_uncertified counts the rows the
 * similarity certificate did not cover; rows_fallback adds those rows to the rows the
 * Euclidean pass over the unit rows recomputed. Pointers, ownership and sizes as
 * knn_search; 1 <= k <= min(N, 1024).
 */
int knn_search_metric(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k, int32_t metric,
                      int32_t* out_idx, float* out_val, const knn_options* opt);

/*
 * k-NN search against a corpus larger than device memory (the paper's Discussion names
 * corpora beyond the GPU's memory as future work). C (N x d) is read in chunks of
 * chunk_rows rows (0: two chunks fit in a quarter of the free device memory); each chunk is
 * searched on the device like knn_search and its answer merged into the running answer
 * by (FP64 direct-difference distance, global index). The indices equal knn_search over
 * the whole corpus; out_dist holds the FP32 rounding of each pair's FP64 distance (a
 * value of the pair alone, whatever the chunking; knn_search reports its FP32 re-rank
 * value, which can differ from it in the last bit). C may be host memory
 * (page-locked memory lets the copy of the next chunk overlap the search of the current
 * one) or device memory; Q and the outputs follow knn_search and must fit on the device.
 * opt->row_threshold must be NULL. opt->stats: counters summed over the chunks
 * (gemm_launches = chunks). Synchronous.
 */
int knn_search_streamed(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k,
                        int64_t chunk_rows, int32_t* out_idx, float* out_dist, const knn_options* opt);

/* The k-NN graph of X by a metric (a point is never its own neighbour); 1 <= k <= N - 1. */
int knng_build_metric(const float* X, int64_t N, int32_t d, int32_t k, int32_t metric, int32_t* out_idx,
                      float* out_val, const knn_options* opt);

/*
 * Quick multi-select alone (Methods, "GPU-based quick multi-select"): the k
 * smallest values of every row of the M x N FP32 matrix D (row stride ldd >= N
 * elements), ascending by (value, column), ties to the lower column. NaN entries
 * are rejected. out_idx (int32), out_val (FP32): M x k. Requires 1 <= k <= N.
 * Few long rows are split into segments selected in parallel and merged (same
 * result). opt->stats (optional): rows and kernel_launches; with KNN_FLAG_TIMING also
 * ms_select (device time of the select kernels) and ms_total (the call's host time).
 */
int knn_select(const float* D, int64_t M, int64_t N, int64_t ldd, int32_t k, int32_t* out_idx, float* out_val,
               const knn_options* opt);

/*
 * Distance matrix alone (Methods, "Distance calculation"): out_D[i*ldd + j] =
 * |c_j|^2 - 2 q_i.c_j (full = 0, the per-row ranking form d') or the squared
 * distance |q_i|^2 + |c_j|^2 - 2 q_i.c_j (full = 1), FP32 SIMT arithmetic.
 */
int knn_distances(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, float* out_D, int64_t ldd,
                  int32_t full, const knn_options* opt);

/*
 * knn_select without any allocation (the paper has no counterpart: this is for
 * callers that cannot let the library allocate -- applications whose device memory
 * is all owned by their own caching allocator or pool, and latency-critical paths
 * that cannot pay cudaMalloc's implicit synchronisation).
 * Same result as knn_select. D, out_idx and out_val must be DEVICE pointers (nothing
 * is staged); stream is a cudaStream_t (NULL = legacy default stream). At most
 * 1048576 rows per call (larger M returns KNN_EINVAL). The only scratch is a fixed
 * 4 MiB device array inside the library, held by every GPU that loads it until exit;
 * the first call on a device looks up that array's address (cudaGetSymbolAddress).
 * All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller. Synchronous like every call: it ends by copying a status
 * word to the host and synchronising the stream. Up to 64 long rows take one CTA per
 * row (knn_select splits them into segments instead, which needs workspace).
 */
int knn_select_noalloc(const float* D, int64_t M, int64_t N, int64_t ldd, int32_t k, int32_t* out_idx,
                       float* out_val, void* stream);

/* One problem of a batch. Pointers follow the conventions above. */
typedef struct knn_problem {
    const float* Q;      /* M x d queries; NULL with exclude_self = 1 means Q = C (a graph) */
    const float* C;      /* N x d corpus */
    int64_t M, N;
    int32_t d, k;
    int32_t exclude_self;/* 1: k-NN graph semantics (requires Q == C or Q == NULL, M == N) */
    int32_t status;      /* out: knn_status of this problem */
    int32_t* out_idx;    /* M x k */
    float* out_dist;     /* M x k */
} knn_problem;

/*
 * Many independent problems of uneven shape in one persistent launch per phase,
 * captured and replayed as a CUDA graph. Per-problem status in probs[i].status.
 * Returns KNN_OK when every problem succeeded, otherwise the first failure.
 */
int knn_search_batched(knn_problem* probs, int32_t count, const knn_options* opt);

/*
 * Learned per-row threshold (the paper has no counterpart). A small network
 * proposes, for each query row, a squared distance below which its k nearest
 * neighbours lie; passed as knn_options.row_threshold it pre-filters candidates, and
 * rows where it cuts into the answer are recomputed without it, so results stay exact.
 *   features (KNN_MLP_FEATURES per row): log |q|^2 and the sorted log squared distances
 *     to KNN_MLP_FEATURES - 1 corpus samples chosen by the caller;
 *   network: KNN_MLP_FEATURES -> KNN_MLP_HIDDEN (ReLU) -> 1, FP32, predicting the log of
 *     the row's exact k-th squared distance from standardised features;
 *   parameters: one FP32 array of knn_mlp_param_count() entries laid out as
 *     W1[H][F] | b1[H] | W2[H] | b2 | mu[F] | sigma[F] | margin
 *     (the first H*F + 2H + 1 are trained; mu/sigma standardise the features; margin is
 *     added to the log prediction to form the threshold).
 * All arrays are device pointers; the caller owns them. Calls are synchronous.
 */
#define KNN_MLP_FEATURES 257
#define KNN_MLP_HIDDEN 128

int32_t knn_mlp_param_count(void);

/* Features of the M query rows Q (M x d) against the samples S (KNN_MLP_FEATURES-1 x d);
 * out_features: M x KNN_MLP_FEATURES. */
int knn_mlp_features(const float* Q, int64_t M, const float* S, int32_t d, float* out_features,
                     const knn_options* opt);

/* Mean squared error 1/n sum (y - t)^2 of the network on (features, targets) and its
 * gradient with respect to the trained parameters (out_grad: H*F + 2H + 1 floats,
 * device; out_loss: host). mu and sigma in params are used as they are. */
int knn_mlp_loss_grad(const float* features, const float* targets, int64_t n, const float* params,
                      double* out_loss, float* out_grad, const knn_options* opt);

/* Trains params in place with Adam (lr, betas 0.9/0.999) on mini-batches of `batch` rows
 * in the given row order for `epochs` epochs, holding out the last round(holdout n) rows;
 * mu/sigma are set from those rows first. The margin is set to the margin_quantile
 * quantile of the held-out residuals t - y (at least 0). out_history (host, optional,
 * `epochs` floats) receives the mean training loss of every epoch. */
int knn_mlp_train(const float* features, const float* targets, int64_t n, float* params, int32_t epochs,
                  int32_t batch, float lr, float holdout, float margin_quantile, float* out_history,
                  const knn_options* opt);

/* Predictions: out_log_kth (optional) receives y; out_threshold (optional) receives
 * exp(y + margin), the squared-distance threshold for knn_options.row_threshold. */
int knn_mlp_predict(const float* features, int64_t n, const float* params, float* out_log_kth,
                    float* out_threshold, const knn_options* opt);

/* Parameter file: magic "KNNMLP01", int32 features, int32 hidden, int32 count, then
 * count FP32 parameters (little-endian). params may be a host or a device pointer;
 * knn_mlp_load rejects a file of another network shape with KNN_EINVAL. */
int knn_mlp_save(const char* path, const float* params);
int knn_mlp_load(const char* path, float* params);

/* Human-readable name of a status code. */
const char* knn_status_string(int status);

/* Message of the last error on the calling thread ("" when none). */
const char* knn_last_error(void);

/* Release the cached workspace of every device this process used. */
void knn_shutdown(void);

/* Library version, e.g. "0.1.0". */
const char* knn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KNN_H */
