/*
 * FP64 brute-force oracle for exact k-nearest-neighbour search and k-NN graphs.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * definition that the GPU engine is checked against. Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it. It shares no
 * code with the CUDA engine.
 *
 * What it computes (Komarov, Dashti, D'Souza, "Fast k-NNG construction with
 * GPU-based quick multi-select", Introduction and Methods):
 *   - the k-NN problem: for each query point, the k corpus points nearest to it;
 *     in the k-NN graph the corpus is the query set and a point is never its own
 *     neighbour (Introduction);
 *   - the Euclidean metric (Methods, "Distance calculation"); the engine reports
 *     SQUARED distances, so the oracle does too. The oracle uses the direct
 *     difference form sum_t (x_t - y_t)^2 rather than the norm expansion the paper
 *     uses on the GPU, so the two sides share no formula;
 *   - the order: ascending (distance, corpus index). The paper does not fix tie
 *     order; the lower index wins here, which makes every answer unique.
 *
 * Precision: inputs are FP32, so every difference x_t - y_t is exact in FP64 and
 * every square has at most 50 significant bits (exact). Only the running sum
 * rounds, with relative error at most d * 2^-53. Integer-valued inputs are exact.
 *
 * Selection: all candidate (distance, index) pairs of a row are sorted with the C
 * library's qsort and the first k are kept. This is the definition itself; it is
 * deliberately not a selection algorithm.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
    double d;
    int64_t j;
} pair_t;

static int pair_cmp(const void* a, const void* b) {
    const pair_t* x = (const pair_t*)a;
    const pair_t* y = (const pair_t*)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    if (x->j < y->j) return -1;
    if (x->j > y->j) return 1;
    return 0;
}

/* Squared Euclidean distance between two d-vectors, direct difference in FP64. */
double oracle_sqdist(const float* x, const float* y, int32_t d) {
    double s = 0.0;
    for (int32_t t = 0; t < d; ++t) {
        double diff = (double)x[t] - (double)y[t];
        s += diff * diff;
    }
    return s;
}

/*
 * k nearest corpus points for selected query rows.
 *   Q: M x d row-major FP32 queries; C: N x d row-major FP32 corpus.
 *   rows[r] (0 <= rows[r] < M) are the query rows to answer (nrows of them).
 *   exclude_self != 0: corpus index j == rows[r] is skipped (k-NN graph, C == Q).
 *   out_idx, out_dist: nrows x k, ascending (distance, index); entries past the
 *   number of available candidates are set to -1 / +inf.
 * Returns 0, or -1 on a bad argument or allocation failure.
 */
int oracle_knn_rows(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k,
                    const int64_t* rows, int64_t nrows, int32_t exclude_self,
                    int64_t* out_idx, double* out_dist) {
    if (!Q || !C || !rows || !out_idx || !out_dist || d < 1 || k < 1 || N < 1 || M < 1) return -1;
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        pair_t* pairs = (pair_t*)malloc((size_t)N * sizeof(pair_t));
        if (!pairs || i < 0 || i >= M) {
            failed = 1;
            free(pairs);
            continue;
        }
        const float* q = Q + (size_t)i * (size_t)d;
        int64_t n = 0;
        for (int64_t j = 0; j < N; ++j) {
            if (exclude_self && j == i) continue;
            pairs[n].d = oracle_sqdist(q, C + (size_t)j * (size_t)d, d);
            pairs[n].j = j;
            ++n;
        }
        qsort(pairs, (size_t)n, sizeof(pair_t), pair_cmp);
        for (int32_t t = 0; t < k; ++t) {
            out_idx[r * k + t] = t < n ? pairs[t].j : -1;
            out_dist[r * k + t] = t < n ? pairs[t].d : __builtin_inf();
        }
        free(pairs);
    }
    return failed ? -1 : 0;
}

/*
 * Cosine and Pearson similarity (Methods, "Distance calculation": the cosine
 * metric x.y / (|x| |y|), and the Pearson metric, the cosine of the vectors
 * centred on the mean of their own entries).
 *
 * FP64 throughout: the mean of a row is sum_t x_t / d; the centred entries
 * x_t - mean; the norm sqrt(sum_t c_t^2); the similarity (sum_t c_t e_t) /
 * (|c| |e|) with c, e the (centred) query and corpus rows. With centered == 0
 * nothing is subtracted and integer-valued inputs give exact dot products and
 * exact squared norms, so the similarity is the correctly rounded quotient of
 * correctly rounded square roots.
 */
static void sim_stats(const float* x, int32_t d, int32_t centered, double* mean, double* norm) {
    double m = 0.0;
    if (centered) {
        for (int32_t t = 0; t < d; ++t) m += (double)x[t];
        m /= (double)d;
    }
    double ss = 0.0;
    for (int32_t t = 0; t < d; ++t) {
        double c = (double)x[t] - m;
        ss += c * c;
    }
    *mean = m;
    *norm = sqrt(ss);
}

/* Similarity of two rows given their means and norms (see above). */
static double sim_pair(const float* x, double mx, double nx, const float* y, double my, double ny, int32_t d) {
    double dot = 0.0;
    for (int32_t t = 0; t < d; ++t) dot += ((double)x[t] - mx) * ((double)y[t] - my);
    return dot / (nx * ny);
}

/* FP64 cosine (centered = 0) or Pearson (centered = 1) similarity of two d-vectors;
 * NaN when either has zero norm. */
double oracle_similarity(const float* x, const float* y, int32_t d, int32_t centered) {
    double mx, nx, my, ny;
    sim_stats(x, d, centered, &mx, &nx);
    sim_stats(y, d, centered, &my, &ny);
    if (nx == 0.0 || ny == 0.0) return __builtin_nan("");
    return sim_pair(x, mx, nx, y, my, ny, d);
}

/*
 * The k most similar corpus points for selected query rows, by cosine
 * (centered = 0) or Pearson (centered = 1) similarity: descending similarity,
 * ties to the lower index. Arguments as oracle_knn_rows; out_sim holds the
 * similarities (-inf past the available candidates). Returns 0, -1 on a bad
 * argument or allocation failure, -2 when a used row has zero (centred) norm.
 */
int oracle_knn_sim_rows(const float* Q, int64_t M, const float* C, int64_t N, int32_t d, int32_t k,
                        int32_t centered, const int64_t* rows, int64_t nrows, int32_t exclude_self,
                        int64_t* out_idx, double* out_sim) {
    if (!Q || !C || !rows || !out_idx || !out_sim || d < 1 || k < 1 || N < 1 || M < 1) return -1;
    double* cm = (double*)malloc((size_t)N * sizeof(double));
    double* cn = (double*)malloc((size_t)N * sizeof(double));
    if (!cm || !cn) {
        free(cm);
        free(cn);
        return -1;
    }
    int zero = 0;
    for (int64_t j = 0; j < N; ++j) {
        sim_stats(C + (size_t)j * (size_t)d, d, centered, &cm[j], &cn[j]);
        if (cn[j] == 0.0) zero = 1;
    }
    int failed = 0;
    if (!zero) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = rows[r];
            pair_t* pairs = (pair_t*)malloc((size_t)N * sizeof(pair_t));
            if (!pairs || i < 0 || i >= M) {
                failed = 1;
                free(pairs);
                continue;
            }
            const float* q = Q + (size_t)i * (size_t)d;
            double qm, qn;
            sim_stats(q, d, centered, &qm, &qn);
            if (qn == 0.0) {
                zero = 1;
                free(pairs);
                continue;
            }
            int64_t n = 0;
            for (int64_t j = 0; j < N; ++j) {
                if (exclude_self && j == i) continue;
                /* ascending -s is descending s; ties keep the lower index first */
                pairs[n].d = -sim_pair(q, qm, qn, C + (size_t)j * (size_t)d, cm[j], cn[j], d);
                pairs[n].j = j;
                ++n;
            }
            qsort(pairs, (size_t)n, sizeof(pair_t), pair_cmp);
            for (int32_t t = 0; t < k; ++t) {
                out_idx[r * k + t] = t < n ? pairs[t].j : -1;
                out_sim[r * k + t] = t < n ? -pairs[t].d : -__builtin_inf();
            }
            free(pairs);
        }
    }
    free(cm);
    free(cn);
    if (zero) return -2;
    return failed ? -1 : 0;
}

/* Number of OpenMP threads the oracle runs on (1 without OpenMP). */
int oracle_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
