/*
 * dkm_oracle.c -- plain FP64 CPU reference for Lloyd's k-means.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the checker that the CUDA path is
 * compared against.  Only the test suite, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load it.  The product library
 * (libdkm) never links, loads or calls anything in this directory, and this
 * file includes nothing from the product.
 *
 * What it computes (Dask-means, arXiv 2412.02244):
 *   - Eq. 1 and Section II-A: k-means minimises the sum of squared errors
 *     sum_j sum_{p in S_j} ||p - c_j||^2, where c_j is the mean of S_j.
 *     Lloyd's algorithm alternates (i) assigning every point to its nearest
 *     centroid (n x k distances) and (ii) resetting each centroid to the mean
 *     of the points assigned to it.
 *   - Section II-B: the accelerated methods (including Dask-means) return the
 *     same result as Lloyd's algorithm, so plain brute-force Lloyd is the
 *     definition that the indexed GPU path must reproduce.
 *   - Algorithm 1 ("Refine centroid": c_j <- sv(j)/|S_j|): the refine step is
 *     the cluster mean.
 *
 * Readings where the paper is silent:
 *   - ties go to the lowest centroid index (scan j = 0..k-1 with strict <);
 *   - an empty cluster keeps its previous centroid (sv/|S| is undefined);
 *   - "converged" = an assignment pass that changes no label;
 *   - max_iter = 0 means: one labelling pass against the initial centroids,
 *     no update, iterations = 0.
 *
 * Arithmetic: inputs are float32 points promoted exactly to double; all
 * distances, sums and means are FP64, evaluated in the order the definition
 * states (no blocking, no reordering).  Points are independent in the
 * assignment, so that loop may run on several host threads (OpenMP); the
 * arithmetic per point is unchanged by that.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* squared Euclidean distance ||p - c||^2 in FP64 (Eq. 1 summand) */
static double sq_dist(const float* p, const double* c, int d) {
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
        double diff = (double)p[t] - c[t];
        s += diff * diff;
    }
    return s;
}

/* nearest and second-nearest centroid of one point; lowest index on ties */
static void nearest_two(const float* p, int d, const double* C, int k,
                        int32_t* a_out, double* d1_out, double* d2_out) {
    double d1 = INFINITY, d2 = INFINITY;
    int32_t a = -1;
    for (int j = 0; j < k; ++j) {
        double s = sq_dist(p, C + (int64_t)j * d, d);
        if (s < d1) {
            d2 = d1;
            d1 = s;
            a = j;
        } else if (s < d2) {
            d2 = s;
        }
    }
    *a_out = a;
    *d1_out = d1;
    *d2_out = d2;
}

/*
 * Assignment step of Lloyd's algorithm (Section II-A): labels[i] =
 * argmin_j ||p_i - c_j||^2.  best[i] / second[i] (nullable) receive the
 * smallest and second-smallest squared distances.
 */
void oracle_assign(const float* pts, int64_t n, int d, const double* C, int k,
                   int32_t* labels, double* best, double* second) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int32_t a;
        double d1, d2;
        nearest_two(pts + i * d, d, C, k, &a, &d1, &d2);
        labels[i] = a;
        if (best) best[i] = d1;
        if (second) second[i] = d2;
    }
}

/* Assignment of a subset of points given by index (sampled parity checks). */
void oracle_assign_subset(const float* pts, int d, const int64_t* idx, int64_t m,
                          const double* C, int k, int32_t* labels, double* best,
                          double* second) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < m; ++s) {
        int32_t a;
        double d1, d2;
        nearest_two(pts + idx[s] * d, d, C, k, &a, &d1, &d2);
        labels[s] = a;
        if (best) best[s] = d1;
        if (second) second[s] = d2;
    }
}

/*
 * Update step (Algorithm 1, "Refine centroid"): c_j = (sum of points with
 * label j) / |S_j| in FP64; an empty cluster keeps C_prev[j].  counts may be
 * NULL.  Returns -1 if a label is out of range, else 0.
 */
int oracle_update(const float* pts, int64_t n, int d, const int32_t* labels, int k,
                  const double* C_prev, double* C_new, int64_t* counts) {
    double* S = (double*)calloc((size_t)k * d, sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)k, sizeof(int64_t));
    if (!S || !cnt) {
        free(S);
        free(cnt);
        return -2;
    }
    for (int64_t i = 0; i < n; ++i) {
        int32_t j = labels[i];
        if (j < 0 || j >= k) {
            free(S);
            free(cnt);
            return -1;
        }
        cnt[j] += 1;
        for (int t = 0; t < d; ++t) S[(int64_t)j * d + t] += (double)pts[i * d + t];
    }
    for (int j = 0; j < k; ++j) {
        for (int t = 0; t < d; ++t) {
            int64_t o = (int64_t)j * d + t;
            C_new[o] = cnt[j] > 0 ? S[o] / (double)cnt[j] : C_prev[o];
        }
        if (counts) counts[j] = cnt[j];
    }
    free(S);
    free(cnt);
    return 0;
}

/* Eq. 1 objective for a given labelling: sum_i ||p_i - c_{label_i}||^2. */
double oracle_sse(const float* pts, int64_t n, int d, const int32_t* labels,
                  const double* C) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += sq_dist(pts + i * d, C + (int64_t)labels[i] * d, d);
    return s;
}

/*
 * Lloyd's algorithm (Algorithm 1 loop with brute-force assignment).
 * One iteration = one assignment pass followed by one update.  With
 * early_stop != 0 the loop ends after the first pass that changes no label
 * (the first pass counts every point as changed).  sse_hist (nullable,
 * length max_iter) receives, after each update, the SSE of that pass's
 * labels against the updated centroids.  Returns 0, or < 0 on error.
 */
int oracle_fit(const float* pts, int64_t n, int d, int k, const double* C0,
               int max_iter, int early_stop, double* C_out, int32_t* labels_out,
               int* iterations_out, double* sse_out, double* sse_hist,
               int64_t* changed_hist) {
    double* C = (double*)malloc((size_t)k * d * sizeof(double));
    double* Cn = (double*)malloc((size_t)k * d * sizeof(double));
    int32_t* lab = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!C || !Cn || !lab) {
        free(C);
        free(Cn);
        free(lab);
        return -2;
    }
    memcpy(C, C0, (size_t)k * d * sizeof(double));
    for (int64_t i = 0; i < n; ++i) labels_out[i] = -1;
    int it = 0;
    if (max_iter <= 0) {
        oracle_assign(pts, n, d, C, k, labels_out, NULL, NULL);
    }
    while (it < max_iter) {
        oracle_assign(pts, n, d, C, k, lab, NULL, NULL);
        int64_t changed = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (lab[i] != labels_out[i]) ++changed;
            labels_out[i] = lab[i];
        }
        ++it;
        int rc = oracle_update(pts, n, d, labels_out, k, C, Cn, NULL);
        if (rc != 0) {
            free(C);
            free(Cn);
            free(lab);
            return rc;
        }
        memcpy(C, Cn, (size_t)k * d * sizeof(double));
        if (sse_hist) sse_hist[it - 1] = oracle_sse(pts, n, d, labels_out, C);
        if (changed_hist) changed_hist[it - 1] = changed;
        if (early_stop && changed == 0) break;
    }
    memcpy(C_out, C, (size_t)k * d * sizeof(double));
    *iterations_out = it;
    *sse_out = oracle_sse(pts, n, d, labels_out, C);
    free(C);
    free(Cn);
    free(lab);
    return 0;
}

/* number of host threads the assignment loop will use (for reporting) */
int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
