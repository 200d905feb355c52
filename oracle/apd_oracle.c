/*
 * FP64 brute-force oracle for anisotropic power diagrams (APDs).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code with
 * the CUDA path.
 *
 * What it computes, in the order of the paper (arXiv 2403.03571):
 *   - pixel centres of the regular grid, eq. (2.6), Section 2.3:
 *       h_d = (hi_d - lo_d) / M_d,  y_d = lo_d + (k_d + 1/2) * h_d
 *     linear pixel id j = k_0 + M_0 * (k_1 + M_1 * k_2) (first axis fastest);
 *   - Algorithm 1: cost C_ij = |y_j - x_i|^2_{A_i} - w_i and H_j in argmin_i C_ij,
 *     the lowest index taken among equal costs (the paper allows any element);
 *       q = sum_a sum_b (d_a * A_ab) * d_b,  d = y - x_i,  a outer, b inner,
 *     accumulated left to right from 0, compiled without FMA contraction;
 *   - per-cell counts m_i and integer moments of the odd pixel coordinates
 *     u = 2k + 1 (y = lo + u h / 2): S1_i = sum u, S2_i = sum u u^T (upper);
 *   - eq. (2.7): g~(W) = sum_i ((v_i - m_i |P|) w_i + sum_{H_j = i} |P| q_ij),
 *     from direct FP64 sums of q (not from the moments);
 *   - eq. (2.8): (grad g)_i ~ v_i - m_i |P|, and the stopping quantity of
 *     Algorithm 2 / eq. (2.5): max_i |v_i - m_i |P|| / v_i;
 *   - the discrete centroids of Algorithm 3: sum_{H_j=i} |P| y_j / (m_i |P|).
 *
 * Threads (OpenMP) split pixels statically; per-thread partial sums are merged
 * in thread order, so results are reproducible for a fixed thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_MEM -6

static int nthreads_or_default(int nt) {
#ifdef _OPENMP
    if (nt <= 0) nt = omp_get_max_threads();
#else
    nt = 1;
#endif
    return nt < 1 ? 1 : nt;
}

static void grid_steps(int dim, const double *lo, const double *hi, const int32_t *res, double *h) {
    for (int d = 0; d < dim; ++d) h[d] = (hi[d] - lo[d]) / (double)res[d];
}

/* pixel centre and odd coordinates of linear id j */
static void pixel_of(int dim, const double *lo, const double *h, const int32_t *res, int64_t j,
                     double *y, int64_t *u) {
    int64_t r = j;
    for (int d = 0; d < dim; ++d) {
        int64_t k = r % res[d];
        r /= res[d];
        y[d] = lo[d] + ((double)k + 0.5) * h[d];
        if (u) u[d] = 2 * k + 1;
    }
}

/* |y - x_i|^2_{A_i}: a outer, b inner */
static double quad_form(int dim, const double *y, const double *xi, const double *Ai) {
    double d[3];
    for (int a = 0; a < dim; ++a) d[a] = y[a] - xi[a];
    double q = 0.0;
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) q = q + d[a] * Ai[a * dim + b] * d[b];
    return q;
}

/* Algorithm 1 for one pixel centre: label, best q, and the relative gap between
 * the two smallest costs, (c2 - c1) / (|q1| + |q2| + |w1| + |w2|) (+inf if n == 1). */
static int32_t assign_one(int dim, const double *y, int32_t n, const double *x, const double *A,
                          const double *w, double *q_best, double *gap) {
    double c1 = INFINITY, c2 = INFINITY, q1 = 0.0, q2 = 0.0, w1 = 0.0, w2 = 0.0;
    int32_t l1 = 0;
    const int dd = dim * dim;
    for (int32_t i = 0; i < n; ++i) {
        double q = quad_form(dim, y, x + (int64_t)i * dim, A + (int64_t)i * dd);
        double c = q - w[i];
        if (c < c1) {
            c2 = c1; q2 = q1; w2 = w1;
            c1 = c; q1 = q; w1 = w[i]; l1 = i;
        } else if (c < c2) {
            c2 = c; q2 = q; w2 = w[i];
        }
    }
    if (q_best) *q_best = q1;
    if (gap) {
        if (n < 2) {
            *gap = INFINITY;
        } else {
            double s = fabs(q1) + fabs(q2) + fabs(w1) + fabs(w2);
            *gap = s > 0.0 ? (c2 - c1) / s : (c2 - c1 > 0.0 ? INFINITY : 0.0);
        }
    }
    return l1;
}

static int check_common(int dim, const int32_t *res, int32_t n) {
    if (dim != 2 && dim != 3) return OR_ERR_ARG;
    if (n < 1) return OR_ERR_ARG;
    for (int d = 0; d < dim; ++d)
        if (res[d] < 1) return OR_ERR_ARG;
    return OR_OK;
}

/* Labels (and optionally relative gaps) for all J pixels. */
int oracle_assign(int32_t dim, const double *lo, const double *hi, const int32_t *res, int32_t n,
                  const double *x, const double *A, const double *w, int32_t *labels, double *gap,
                  int32_t nthreads) {
    if (check_common(dim, res, n) || !labels) return OR_ERR_ARG;
    double h[3];
    grid_steps(dim, lo, hi, res, h);
    int64_t J = 1;
    for (int d = 0; d < dim; ++d) J *= res[d];
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int64_t j = 0; j < J; ++j) {
        double y[3];
        pixel_of(dim, lo, h, res, j, y, NULL);
        labels[j] = assign_one(dim, y, n, x, A, w, NULL, gap ? gap + j : NULL);
    }
    return OR_OK;
}

/* Labels (and gaps) for a list of pixel ids only. */
int oracle_assign_ids(int32_t dim, const double *lo, const double *hi, const int32_t *res, int32_t n,
                      const double *x, const double *A, const double *w, const int64_t *ids,
                      int64_t count, int32_t *labels, double *gap, int32_t nthreads) {
    if (check_common(dim, res, n) || (!ids && count > 0) || (!labels && count > 0)) return OR_ERR_ARG;
    double h[3];
    grid_steps(dim, lo, hi, res, h);
    int64_t J = 1;
    for (int d = 0; d < dim; ++d) J *= res[d];
    for (int64_t t = 0; t < count; ++t)
        if (ids[t] < 0 || ids[t] >= J) return OR_ERR_ARG;
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int64_t t = 0; t < count; ++t) {
        double y[3];
        pixel_of(dim, lo, h, res, ids[t], y, NULL);
        labels[t] = assign_one(dim, y, n, x, A, w, NULL, gap ? gap + t : NULL);
    }
    return OR_OK;
}

/* Integer moments per cell from labels: out[i*K + 0] = m_i, then S1 (dim
 * entries), then the upper triangle of S2 row by row; K = 1 + dim + dim(dim+1)/2. */
int oracle_moments(int32_t dim, const int32_t *res, int32_t n, const int32_t *labels, int64_t *out,
                   int32_t nthreads) {
    if (check_common(dim, res, n) || !labels || !out) return OR_ERR_ARG;
    const int K = 1 + dim + dim * (dim + 1) / 2;
    int64_t J = 1;
    for (int d = 0; d < dim; ++d) J *= res[d];
    int nt = nthreads_or_default(nthreads);
    int64_t *part = (int64_t *)calloc((size_t)nt * (size_t)n * K, sizeof(int64_t));
    if (!part) return OR_ERR_MEM;
    int bad = 0;
#pragma omp parallel num_threads(nt) reduction(| : bad)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        int64_t *p = part + (size_t)t * n * K;
#pragma omp for schedule(static)
        for (int64_t j = 0; j < J; ++j) {
            int32_t l = labels[j];
            if (l < 0 || l >= n) { bad = 1; continue; }
            int64_t u[3];
            int64_t r = j;
            for (int d = 0; d < dim; ++d) { u[d] = 2 * (r % res[d]) + 1; r /= res[d]; }
            int64_t *o = p + (size_t)l * K;
            o[0] += 1;
            for (int d = 0; d < dim; ++d) o[1 + d] += u[d];
            int s = 1 + dim;
            for (int a = 0; a < dim; ++a)
                for (int b = a; b < dim; ++b) o[s++] += u[a] * u[b];
        }
    }
    memset(out, 0, sizeof(int64_t) * (size_t)n * K);
    for (int t = 0; t < nt; ++t)
        for (int64_t e = 0; e < (int64_t)n * K; ++e) out[e] += part[(size_t)t * n * K + e];
    free(part);
    return bad ? OR_ERR_ARG : OR_OK;
}

/* The same integer moments over a listed subset of pixels: labels[t] is the
 * label of pixel ids[t] (full-grid linear id), and u = 2k + 1 uses the full
 * grid's indices k, so the moments of disjoint subsets add up to those of
 * their union. */
int oracle_moments_ids(int32_t dim, const int32_t *res, int32_t n, const int64_t *ids, int64_t count,
                       const int32_t *labels, int64_t *out, int32_t nthreads) {
    if (check_common(dim, res, n) || !ids || !labels || !out || count < 0) return OR_ERR_ARG;
    const int K = 1 + dim + dim * (dim + 1) / 2;
    int64_t J = 1;
    for (int d = 0; d < dim; ++d) J *= res[d];
    int nt = nthreads_or_default(nthreads);
    int64_t *part = (int64_t *)calloc((size_t)nt * (size_t)n * K, sizeof(int64_t));
    if (!part) return OR_ERR_MEM;
    int bad = 0;
#pragma omp parallel num_threads(nt) reduction(| : bad)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        int64_t *p = part + (size_t)t * n * K;
#pragma omp for schedule(static)
        for (int64_t e = 0; e < count; ++e) {
            int32_t l = labels[e];
            int64_t j = ids[e];
            if (l < 0 || l >= n || j < 0 || j >= J) { bad = 1; continue; }
            int64_t u[3];
            int64_t r = j;
            for (int d = 0; d < dim; ++d) { u[d] = 2 * (r % res[d]) + 1; r /= res[d]; }
            int64_t *o = p + (size_t)l * K;
            o[0] += 1;
            for (int d = 0; d < dim; ++d) o[1 + d] += u[d];
            int s = 1 + dim;
            for (int a = 0; a < dim; ++a)
                for (int b = a; b < dim; ++b) o[s++] += u[a] * u[b];
        }
    }
    memset(out, 0, sizeof(int64_t) * (size_t)n * K);
    for (int t = 0; t < nt; ++t)
        for (int64_t e = 0; e < (int64_t)n * K; ++e) out[e] += part[(size_t)t * n * K + e];
    free(part);
    return bad ? OR_ERR_ARG : OR_OK;
}

/* Per-cell direct sums for a given labelling: count m_i, cost sum
 * Qsum_i = sum_{H_j=i} q_ij, and coordinate sums Ysum_i = sum_{H_j=i} y_j. */
static int cell_sums(int32_t dim, const double *lo, const double *hi, const int32_t *res, int32_t n,
                     const double *x, const double *A, const int32_t *labels, int64_t *m,
                     double *qsum, double *ysum, int nt) {
    double h[3];
    grid_steps(dim, lo, hi, res, h);
    int64_t J = 1;
    for (int d = 0; d < dim; ++d) J *= res[d];
    const int dd = dim * dim;
    int64_t *pm = (int64_t *)calloc((size_t)nt * n, sizeof(int64_t));
    double *pq = (double *)calloc((size_t)nt * n, sizeof(double));
    double *py = (double *)calloc((size_t)nt * n * dim, sizeof(double));
    if (!pm || !pq || !py) { free(pm); free(pq); free(py); return OR_ERR_MEM; }
    int bad = 0;
#pragma omp parallel num_threads(nt) reduction(| : bad)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
#pragma omp for schedule(static)
        for (int64_t j = 0; j < J; ++j) {
            int32_t l = labels[j];
            if (l < 0 || l >= n) { bad = 1; continue; }
            double y[3];
            pixel_of(dim, lo, h, res, j, y, NULL);
            pm[(size_t)t * n + l] += 1;
            pq[(size_t)t * n + l] += quad_form(dim, y, x + (int64_t)l * dim, A + (int64_t)l * dd);
            for (int d = 0; d < dim; ++d) py[((size_t)t * n + l) * dim + d] += y[d];
        }
    }
    for (int32_t i = 0; i < n; ++i) {
        int64_t mm = 0;
        double qq = 0.0;
        double yy[3] = {0.0, 0.0, 0.0};
        for (int t = 0; t < nt; ++t) {
            mm += pm[(size_t)t * n + i];
            qq += pq[(size_t)t * n + i];
            for (int d = 0; d < dim; ++d) yy[d] += py[((size_t)t * n + i) * dim + d];
        }
        if (m) m[i] = mm;
        if (qsum) qsum[i] = qq;
        if (ysum)
            for (int d = 0; d < dim; ++d) ysum[(size_t)i * dim + d] = yy[d];
    }
    free(pm); free(pq); free(py);
    return bad ? OR_ERR_ARG : OR_OK;
}

/* Dual value and approximate gradient for a given labelling, eqs. (2.7)-(2.8).
 * out: g[0], grad[n], max_rel_err[0]; m (optional) receives the counts and
 * qsum (optional) the per-cell cost sums. */
int oracle_dual_from_labels(int32_t dim, const double *lo, const double *hi, const int32_t *res,
                            int32_t n, const double *x, const double *A, const double *w,
                            const double *v, const int32_t *labels, double *g, double *grad,
                            double *max_rel_err, int64_t *m_out, double *qsum_out,
                            int32_t nthreads) {
    if (check_common(dim, res, n) || !labels || !v || !w) return OR_ERR_ARG;
    int nt = nthreads_or_default(nthreads);
    double h[3];
    grid_steps(dim, lo, hi, res, h);
    double P = 1.0;
    for (int d = 0; d < dim; ++d) P *= h[d];
    int64_t *m = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *qs = (double *)malloc(sizeof(double) * (size_t)n);
    if (!m || !qs) { free(m); free(qs); return OR_ERR_MEM; }
    int rc = cell_sums(dim, lo, hi, res, n, x, A, labels, m, qs, NULL, nt);
    if (rc) { free(m); free(qs); return rc; }
    double gv = 0.0, err = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        double vol = (double)m[i] * P;
        double gi = v[i] - vol;
        gv += gi * w[i] + P * qs[i];
        if (grad) grad[i] = gi;
        double e = fabs(gi) / v[i];
        if (e > err) err = e;
        if (m_out) m_out[i] = m[i];
        if (qsum_out) qsum_out[i] = qs[i];
    }
    if (g) *g = gv;
    if (max_rel_err) *max_rel_err = err;
    free(m); free(qs);
    return OR_OK;
}

/* Discrete centroids of Algorithm 3 for a labelling; empty cells keep x_i. */
int oracle_centroids(int32_t dim, const double *lo, const double *hi, const int32_t *res, int32_t n,
                     const double *x, const int32_t *labels, double *x_out, int32_t nthreads) {
    if (check_common(dim, res, n) || !labels || !x || !x_out) return OR_ERR_ARG;
    int nt = nthreads_or_default(nthreads);
    double h[3];
    grid_steps(dim, lo, hi, res, h);
    double P = 1.0;
    for (int d = 0; d < dim; ++d) P *= h[d];
    int64_t *m = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *ys = (double *)malloc(sizeof(double) * (size_t)n * dim);
    double *Aid = (double *)calloc((size_t)n * dim * dim, sizeof(double));
    if (!m || !ys || !Aid) { free(m); free(ys); free(Aid); return OR_ERR_MEM; }
    int rc = cell_sums(dim, lo, hi, res, n, x, Aid, labels, m, NULL, ys, nt);
    if (rc) { free(m); free(ys); free(Aid); return rc; }
    for (int32_t i = 0; i < n; ++i)
        for (int d = 0; d < dim; ++d) {
            size_t e = (size_t)i * dim + d;
            /* sum |P| y_j / sum |P|, as printed in Algorithm 3 */
            x_out[e] = m[i] > 0 ? (P * ys[e]) / (P * (double)m[i]) : x[e];
        }
    free(m); free(ys); free(Aid);
    return OR_OK;
}

/* Cost of one (pixel, seed) pair, exposed for tests. */
double oracle_cost(int32_t dim, const double *y, const double *xi, const double *Ai, double wi) {
    return quad_form(dim, y, xi, Ai) - wi;
}

int oracle_max_threads(void) { return nthreads_or_default(0); }
