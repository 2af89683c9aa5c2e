/*
 * Plain FP64 CPU oracle for the leave-one-out cross-validated log-likelihood
 * of the double-kernel (Nadaraya-Watson) conditional density estimator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the test suite, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * Conventions (Holmes, Gray & Isbell, Sec. 2 and Sec. 3):
 *   h1 = bandwidth on x (d dimensions), h2 = bandwidth on y (1 dimension);
 *   K_h(t) = h^{-d} K(t/h) with K the standard normal density (Sec. 2 scaling).
 *   A_j(h1,h2) = sum_{i != j} K_h1(|x_j - x_i|) K_h2(y_j - y_i)     (Sec. 3.2)
 *   B_j(h1)    = sum_{i != j} K_h1(|x_j - x_i|)                     (Sec. 3.2)
 *   ell_j      = ln A_j - ln B_j = ln fhat^{-j}(y_j | x_j)          (Eq. 1)
 *   L_cond     = sum_j ell_j                (conditional LOO log-likelihood)
 *   L_eq3      = (1/n) sum_j ln(fhat^{-j}(y_j|x_j) fhat^{-j}(x_j))   (Eq. 3)
 *              = (1/n) sum_j ln A_j - ln(n-1)                       (Sec. 3.2)
 * Second kernel family (kernel = 1): the radial Epanechnikov kernel that the
 * paper uses in all its experiments (Sec. 4),
 *   K(t) = c_d (1 - |t|^2) for |t| < 1, 0 otherwise,  c_d = (d + 2) / (2 V_d),
 *   V_d = pi^{d/2} / Gamma(d/2 + 1) (volume of the unit d-ball),
 * with the same h^{-d} scaling.  Its sums are plain sums of bounded terms.
 * Compact support makes exact zeros possible: A_j = 0 gives ell_j = -inf
 * (the paper's divergence at small bandwidths, Sec. 4.1), and so does an
 * empty x-neighbourhood (B_j = 0, where Eq. 1 is 0/0).
 * Every Gaussian sum over i is evaluated with a log-sum-exp (max, then sum of
 * shifted exponentials) so that no bandwidth underflows; every loop is a
 * straight loop over all i != j (exclusion by index).  Rows j are split across threads;
 * sums over j are Neumaier-compensated in a fixed block order, so results do
 * not depend on the thread count.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LN_SQRT_2PI 0.91893853320467274178 /* ln sqrt(2 pi) */
#define ROW_BLOCK 256

typedef struct { double s, c; } neumaier_t;

static void nm_add(neumaier_t *a, double v) {
    if (isinf(v) || isinf(a->s)) {  /* -inf terms (Epanechnikov): no compensation */
        a->s += v;
        return;
    }
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static double nm_val(const neumaier_t *a) { return a->s + a->c; }

/* Standardisation used on the paper's data (Sec. 4): each x dimension is
 * centred and divided by its sample standard deviation (ddof = 1).
 * x is N x d row-major (FP32 values widened to FP64).  Returns -1 when a
 * dimension has zero spread. */
int oracle_standardize(const double *x, int64_t N, int d, double *out) {
    for (int c = 0; c < d; ++c) {
        neumaier_t m = {0, 0};
        for (int64_t i = 0; i < N; ++i) nm_add(&m, x[i * d + c]);
        double mean = nm_val(&m) / (double)N;
        neumaier_t v = {0, 0};
        for (int64_t i = 0; i < N; ++i) {
            double t = x[i * d + c] - mean;
            nm_add(&v, t * t);
        }
        double sd = sqrt(nm_val(&v) / (double)(N - 1));
        if (!(sd > 0.0)) return -1;
        for (int64_t i = 0; i < N; ++i) out[i * d + c] = (x[i * d + c] - mean) / sd;
    }
    return 0;
}

static double sqdist(const double *a, const double *b, int d) {
    double s = 0.0;
    for (int c = 0; c < d; ++c) {
        double t = a[c] - b[c];
        s += t * t;
    }
    return s;
}

/* ln c_d of the radial Epanechnikov kernel in d dimensions. */
static double epan_log_cd(int d) {
    return log(d + 2.0) - log(2.0) - 0.5 * d * log(M_PI) + lgamma(0.5 * d + 1.0);
}

/* Epanechnikov profile (1 - t2/h^2)_+ (no normalisation). */
static double epan_prof(double t2, double h) {
    const double v = 1.0 - t2 / (h * h);
    return v > 0.0 ? v : 0.0;
}

/* ln sum_{i != j} exp(e_i), by max then shifted sum. */
static double lse_excl(const double *e, int64_t N, int64_t j) {
    double m = -INFINITY;
    for (int64_t i = 0; i < N; ++i)
        if (i != j && e[i] > m) m = e[i];
    if (m == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i)
        if (i != j) s += exp(e[i] - m);
    return m + log(s);
}

/* ------------------------------------------------------------------ */
/* Per-row LOO log terms                                               */
/* ------------------------------------------------------------------ */
typedef struct {
    const double *x, *y, *h1, *h2;
    int64_t N;
    int d, G1, G2;
    const int64_t *rows;      /* NULL: all rows */
    int64_t n_rows;
    double *ell;              /* optional: n_rows x G1 x G2 */
    double *lnA;              /* optional: n_rows x G1 x G2 */
    neumaier_t *blk_cond;     /* optional: n_blocks x G1 x G2 */
    neumaier_t *blk_lnA;      /* optional: n_blocks x G1 x G2 */
    int64_t block;            /* rows per work item (fixed: sums do not depend on threads) */
    int kernel;               /* 0 Gaussian, 1 Epanechnikov */
    int64_t next_block;
    pthread_mutex_t mu;
} rows_job_t;

/* Epanechnikov row terms: plain sums of K_h1 K_h2 and of K_h1 over i != j. */
static void row_terms_epan(const rows_job_t *J, int64_t j, const double *dx2, const double *dy2,
                           double *ell_out, double *lnA_out) {
    const int d = J->d;
    const double lcd = epan_log_cd(d), lc1 = epan_log_cd(1);
    for (int k = 0; k < J->G1; ++k) {
        const double h1 = J->h1[k];
        double B = 0.0;
        for (int64_t i = 0; i < J->N; ++i)
            if (i != j) B += epan_prof(dx2[i], h1);
        const double lnB = log(B) + lcd - d * log(h1);
        for (int l = 0; l < J->G2; ++l) {
            const double h2 = J->h2[l];
            double A = 0.0;
            for (int64_t i = 0; i < J->N; ++i)
                if (i != j) A += epan_prof(dx2[i], h1) * epan_prof(dy2[i], h2);
            const double lnA = log(A) + lcd - d * log(h1) + lc1 - log(h2);
            ell_out[k * J->G2 + l] = B > 0.0 ? lnA - lnB : -INFINITY;
            lnA_out[k * J->G2 + l] = lnA;
        }
    }
}

static void row_terms(const rows_job_t *J, int64_t j, double *dx2, double *dy2, double *e,
                      double *ell_out, double *lnA_out) {
    const int d = J->d;
    for (int64_t i = 0; i < J->N; ++i) {
        dx2[i] = sqdist(J->x + j * d, J->x + i * d, d);
        double t = J->y[j] - J->y[i];
        dy2[i] = t * t;
    }
    if (J->kernel == 1) {
        row_terms_epan(J, j, dx2, dy2, ell_out, lnA_out);
        return;
    }
    for (int k = 0; k < J->G1; ++k) {
        const double h1 = J->h1[k];
        for (int64_t i = 0; i < J->N; ++i) e[i] = -dx2[i] / (2.0 * h1 * h1);
        /* ln B_j = ln sum K_h1 */
        const double lnB = lse_excl(e, J->N, j) - d * (LN_SQRT_2PI + log(h1));
        for (int l = 0; l < J->G2; ++l) {
            const double h2 = J->h2[l];
            for (int64_t i = 0; i < J->N; ++i)
                e[i] = -dx2[i] / (2.0 * h1 * h1) - dy2[i] / (2.0 * h2 * h2);
            const double lnA = lse_excl(e, J->N, j) - d * (LN_SQRT_2PI + log(h1))
                               - (LN_SQRT_2PI + log(h2));
            ell_out[k * J->G2 + l] = lnA - lnB;
            lnA_out[k * J->G2 + l] = lnA;
        }
    }
}

static void *rows_worker(void *arg) {
    rows_job_t *J = (rows_job_t *)arg;
    const int64_t G = (int64_t)J->G1 * J->G2;
    double *dx2 = malloc(sizeof(double) * J->N);
    double *dy2 = malloc(sizeof(double) * J->N);
    double *e = malloc(sizeof(double) * J->N);
    double *ell = malloc(sizeof(double) * G);
    double *lnA = malloc(sizeof(double) * G);
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t b = J->next_block++;
        pthread_mutex_unlock(&J->mu);
        int64_t r0 = b * J->block;
        if (r0 >= J->n_rows) break;
        int64_t r1 = r0 + J->block < J->n_rows ? r0 + J->block : J->n_rows;
        for (int64_t r = r0; r < r1; ++r) {
            int64_t j = J->rows ? J->rows[r] : r;
            row_terms(J, j, dx2, dy2, e, ell, lnA);
            if (J->ell) memcpy(J->ell + r * G, ell, sizeof(double) * G);
            if (J->lnA) memcpy(J->lnA + r * G, lnA, sizeof(double) * G);
            if (J->blk_cond)
                for (int64_t c = 0; c < G; ++c) {
                    nm_add(&J->blk_cond[b * G + c], ell[c]);
                    nm_add(&J->blk_lnA[b * G + c], lnA[c]);
                }
        }
    }
    free(dx2); free(dy2); free(e); free(ell); free(lnA);
    return NULL;
}

static void run_rows(rows_job_t *J, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    pthread_mutex_init(&J->mu, NULL);
    J->next_block = 0;
    pthread_t *th = malloc(sizeof(pthread_t) * n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, rows_worker, J);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J->mu);
}

/* ell_j(k,l) and ln A_j(k,l) for the listed rows (rows == NULL: 0..n_rows-1).
 * Outputs are n_rows x G1 x G2, row-major with h1 major. */
void oracle_loo_rows(const double *x, const double *y, int64_t N, int d,
                     const double *h1, int G1, const double *h2, int G2,
                     const int64_t *rows, int64_t n_rows, double *ell, double *lnA,
                     int n_threads, int kernel) {
    rows_job_t J;
    memset(&J, 0, sizeof(J));
    J.kernel = kernel;
    J.x = x; J.y = y; J.h1 = h1; J.h2 = h2; J.N = N; J.d = d; J.G1 = G1; J.G2 = G2;
    J.rows = rows; J.n_rows = n_rows; J.ell = ell; J.lnA = lnA;
    J.block = 1;
    run_rows(&J, n_threads);
}

/* Whole-grid scores: L_cond[k][l] = sum_j ell_j, L_eq3[k][l] = (1/N) sum_j ln A_j - ln(N-1). */
void oracle_loo_grid(const double *x, const double *y, int64_t N, int d,
                     const double *h1, int G1, const double *h2, int G2,
                     double *L_cond, double *L_eq3, int n_threads, int kernel) {
    const int64_t G = (int64_t)G1 * G2;
    const int64_t n_blocks = (N + ROW_BLOCK - 1) / ROW_BLOCK;
    rows_job_t J;
    memset(&J, 0, sizeof(J));
    J.kernel = kernel;
    J.x = x; J.y = y; J.h1 = h1; J.h2 = h2; J.N = N; J.d = d; J.G1 = G1; J.G2 = G2;
    J.rows = NULL; J.n_rows = N;
    J.block = ROW_BLOCK;
    J.blk_cond = calloc((size_t)(n_blocks * G), sizeof(neumaier_t));
    J.blk_lnA = calloc((size_t)(n_blocks * G), sizeof(neumaier_t));
    run_rows(&J, n_threads);
    for (int64_t c = 0; c < G; ++c) {
        neumaier_t a = {0, 0}, b = {0, 0};
        for (int64_t bl = 0; bl < n_blocks; ++bl) {
            nm_add(&a, nm_val(&J.blk_cond[bl * G + c]));
            nm_add(&b, nm_val(&J.blk_lnA[bl * G + c]));
        }
        L_cond[c] = nm_val(&a);
        L_eq3[c] = nm_val(&b) / (double)N - log((double)(N - 1));
    }
    free(J.blk_cond);
    free(J.blk_lnA);
}

/* ------------------------------------------------------------------ */
/* Gradient of L_cond with respect to (ln h1, ln h2) at one bandwidth  */
/* ------------------------------------------------------------------ */
/* Derivation (the paper gives none; it follows from the Gaussian K):
 *   d ln K_h1(r)/d ln h1 = r^2/h1^2 - d,   d ln K_h2(t)/d ln h2 = t^2/h2^2 - 1,
 *   d ell_j/d ln h1 = (E_Aj[dx2] - E_Bj[dx2]) / h1^2,
 *   d ell_j/d ln h2 = E_Aj[dy2] / h2^2 - 1,
 * where E_Aj weights i by K_h1 K_h2 and E_Bj by K_h1 (i != j). */
typedef struct {
    const double *x, *y;
    int64_t N;
    int d;
    double h1, h2;
    const int64_t *rows;
    int64_t n_rows;
    double *row_out;          /* optional n_rows x 3: ell, d/dlnh1, d/dlnh2 */
    neumaier_t *blk;          /* n_blocks x 3 */
    int kernel;               /* 0 Gaussian, 1 Epanechnikov */
    int64_t next_block;
    pthread_mutex_t mu;
} grad_job_t;

/* Epanechnikov: with u = (1 - dx2/h1^2)_+ and w = (1 - dy2/h2^2)_+,
 *   d K_h1/d ln h1 = c_d h1^{-d} (2 dx2/h1^2 [dx2 < h1^2] - d u),
 *   d K_h2/d ln h2 = c_1 h2^{-1} (2 dy2/h2^2 [dy2 < h2^2] - w),
 * so, with v = 2 dx2/h1^2 [dx2 < h1^2] and z = 2 dy2/h2^2 [dy2 < h2^2],
 *   d ell_j/d ln h1 = sum v w / sum u w - sum v / sum u,
 *   d ell_j/d ln h2 = sum u z / sum u w - 1.
 * A row with A_j = 0 has ell_j = -inf and contributes 0 to both derivatives. */
static void grad_row_epan(const grad_job_t *J, int64_t j, const double *dx2, const double *dy2,
                          double out[3]) {
    const int d = J->d;
    const double h1 = J->h1, h2 = J->h2;
    double sA = 0, sAv = 0, sAz = 0, sB = 0, sBv = 0;
    for (int64_t i = 0; i < J->N; ++i) {
        if (i == j) continue;
        const double u = epan_prof(dx2[i], h1), w = epan_prof(dy2[i], h2);
        const double v = dx2[i] < h1 * h1 ? 2.0 * dx2[i] / (h1 * h1) : 0.0;
        const double z = dy2[i] < h2 * h2 ? 2.0 * dy2[i] / (h2 * h2) : 0.0;
        sA += u * w; sAv += v * w; sAz += u * z;
        sB += u; sBv += v;
    }
    const double lnA = log(sA) + epan_log_cd(d) - d * log(h1) + epan_log_cd(1) - log(h2);
    const double lnB = log(sB) + epan_log_cd(d) - d * log(h1);
    out[0] = sB > 0.0 ? lnA - lnB : -INFINITY;
    out[1] = sA > 0.0 ? sAv / sA - sBv / sB : 0.0;
    out[2] = sA > 0.0 ? sAz / sA - 1.0 : 0.0;
}

static void grad_row(const grad_job_t *J, int64_t j, double *dx2, double *dy2, double out[3]) {
    const int d = J->d;
    const double a1 = 1.0 / (2.0 * J->h1 * J->h1), a2 = 1.0 / (2.0 * J->h2 * J->h2);
    double mA = -INFINITY, mB = -INFINITY;
    if (J->kernel == 1) {
        for (int64_t i = 0; i < J->N; ++i) {
            dx2[i] = sqdist(J->x + j * d, J->x + i * d, d);
            double t = J->y[j] - J->y[i];
            dy2[i] = t * t;
        }
        grad_row_epan(J, j, dx2, dy2, out);
        return;
    }
    for (int64_t i = 0; i < J->N; ++i) {
        dx2[i] = sqdist(J->x + j * d, J->x + i * d, d);
        double t = J->y[j] - J->y[i];
        dy2[i] = t * t;
        if (i == j) continue;
        double eA = -a1 * dx2[i] - a2 * dy2[i], eB = -a1 * dx2[i];
        if (eA > mA) mA = eA;
        if (eB > mB) mB = eB;
    }
    double sA = 0, sAx = 0, sAy = 0, sB = 0, sBx = 0;
    for (int64_t i = 0; i < J->N; ++i) {
        if (i == j) continue;
        double wA = exp(-a1 * dx2[i] - a2 * dy2[i] - mA);
        double wB = exp(-a1 * dx2[i] - mB);
        sA += wA; sAx += wA * dx2[i]; sAy += wA * dy2[i];
        sB += wB; sBx += wB * dx2[i];
    }
    double lnA = mA + log(sA) - d * (LN_SQRT_2PI + log(J->h1)) - (LN_SQRT_2PI + log(J->h2));
    double lnB = mB + log(sB) - d * (LN_SQRT_2PI + log(J->h1));
    out[0] = lnA - lnB;
    out[1] = (sAx / sA - sBx / sB) / (J->h1 * J->h1);
    out[2] = (sAy / sA) / (J->h2 * J->h2) - 1.0;
}

static void *grad_worker(void *arg) {
    grad_job_t *J = (grad_job_t *)arg;
    double *dx2 = malloc(sizeof(double) * J->N);
    double *dy2 = malloc(sizeof(double) * J->N);
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t b = J->next_block++;
        pthread_mutex_unlock(&J->mu);
        int64_t r0 = b * ROW_BLOCK;
        if (r0 >= J->n_rows) break;
        int64_t r1 = r0 + ROW_BLOCK < J->n_rows ? r0 + ROW_BLOCK : J->n_rows;
        for (int64_t r = r0; r < r1; ++r) {
            double o[3];
            grad_row(J, J->rows ? J->rows[r] : r, dx2, dy2, o);
            if (J->row_out) memcpy(J->row_out + 3 * r, o, sizeof(o));
            for (int c = 0; c < 3; ++c) nm_add(&J->blk[b * 3 + c], o[c]);
        }
    }
    free(dx2); free(dy2);
    return NULL;
}

/* L_cond and its gradient (d/d ln h1, d/d ln h2) over the listed rows
 * (rows == NULL: all N rows).  out3 = {L, dL/dlnh1, dL/dlnh2}. */
void oracle_grad(const double *x, const double *y, int64_t N, int d, double h1, double h2,
                 const int64_t *rows, int64_t n_rows, double *row_out, double *out3,
                 int n_threads, int kernel) {
    grad_job_t J;
    memset(&J, 0, sizeof(J));
    J.kernel = kernel;
    J.x = x; J.y = y; J.N = N; J.d = d; J.h1 = h1; J.h2 = h2;
    J.rows = rows; J.n_rows = n_rows; J.row_out = row_out;
    const int64_t n_blocks = (n_rows + ROW_BLOCK - 1) / ROW_BLOCK;
    J.blk = calloc((size_t)(n_blocks * 3 + 3), sizeof(neumaier_t));
    pthread_mutex_init(&J.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = malloc(sizeof(pthread_t) * n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, grad_worker, &J);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
    for (int c = 0; c < 3; ++c) {
        neumaier_t a = {0, 0};
        for (int64_t b = 0; b < n_blocks; ++b) nm_add(&a, nm_val(&J.blk[b * 3 + c]));
        out3[c] = nm_val(&a);
    }
    free(J.blk);
}

/* ------------------------------------------------------------------ */
/* Conditional density at query points (Eq. 1, no leave-one-out)       */
/* ------------------------------------------------------------------ */
typedef struct {
    const double *x, *y, *xq, *yg;
    int64_t N, Q;
    int d, G;
    double h1, h2;
    double *f;
    int kernel;               /* 0 Gaussian, 1 Epanechnikov */
    int64_t next;
    pthread_mutex_t mu;
} dens_job_t;

/* Epanechnikov: plain sums; a query with no x-neighbour inside h1 (Eq. 1 is
 * 0/0 there) gets f = 0 on the whole y grid. */
static void dens_query_epan(const dens_job_t *J, int64_t q, double *ex) {
    const double lc1 = epan_log_cd(1);
    double B = 0.0;
    for (int64_t i = 0; i < J->N; ++i) {
        ex[i] = epan_prof(sqdist(J->xq + q * J->d, J->x + i * J->d, J->d), J->h1);
        B += ex[i];
    }
    for (int g = 0; g < J->G; ++g) {
        double A = 0.0;
        for (int64_t i = 0; i < J->N; ++i) {
            const double t = J->yg[g] - J->y[i];
            A += ex[i] * epan_prof(t * t, J->h2);
        }
        J->f[q * J->G + g] = B > 0.0 ? A / B * exp(lc1 - log(J->h2)) : 0.0;
    }
}

static void *dens_worker(void *arg) {
    dens_job_t *J = (dens_job_t *)arg;
    double *ex = malloc(sizeof(double) * J->N);
    double *e = malloc(sizeof(double) * J->N);
    const double a1 = 1.0 / (2.0 * J->h1 * J->h1), a2 = 1.0 / (2.0 * J->h2 * J->h2);
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t q = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (q >= J->Q) break;
        if (J->kernel == 1) {
            dens_query_epan(J, q, ex);
            continue;
        }
        double mB = -INFINITY;
        for (int64_t i = 0; i < J->N; ++i) {
            ex[i] = -a1 * sqdist(J->xq + q * J->d, J->x + i * J->d, J->d);
            if (ex[i] > mB) mB = ex[i];
        }
        double sB = 0;
        for (int64_t i = 0; i < J->N; ++i) sB += exp(ex[i] - mB);
        const double lnB = mB + log(sB);
        for (int g = 0; g < J->G; ++g) {
            double mA = -INFINITY;
            for (int64_t i = 0; i < J->N; ++i) {
                double t = J->yg[g] - J->y[i];
                e[i] = ex[i] - a2 * t * t;
                if (e[i] > mA) mA = e[i];
            }
            double sA = 0;
            for (int64_t i = 0; i < J->N; ++i) sA += exp(e[i] - mA);
            double lnf = mA + log(sA) - lnB - (LN_SQRT_2PI + log(J->h2));
            J->f[q * J->G + g] = exp(lnf);
        }
    }
    free(ex); free(e);
    return NULL;
}

/* f[q][g] = fhat(yg[g] | xq[q]) of Eq. 1 over all N points (kernel 0 Gaussian,
 * 1 Epanechnikov). */
void oracle_density(const double *x, const double *y, int64_t N, int d, double h1, double h2,
                    const double *xq, int64_t Q, const double *yg, int G, double *f,
                    int n_threads, int kernel) {
    dens_job_t J;
    memset(&J, 0, sizeof(J));
    J.kernel = kernel;
    J.x = x; J.y = y; J.xq = xq; J.yg = yg; J.N = N; J.Q = Q; J.d = d; J.G = G;
    J.h1 = h1; J.h2 = h2; J.f = f;
    pthread_mutex_init(&J.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = malloc(sizeof(pthread_t) * n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, dens_worker, &J);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
}

/* ------------------------------------------------------------------ */
/* Products of the conditional density at query points (Sec. 4.2)     */
/* ------------------------------------------------------------------ */
/* With x weights K_h1(x_q - x_i) (Eq. 1), at each query q:
 *   mean[q] = E[y | x_q] = sum_i K_h1 y_i / sum_i K_h1 (the y kernel is symmetric),
 *   fat[q]  = fhat(yq[q] | x_q),
 *   F[q][g] = P(y <= yg[g] | x_q) = sum_i K_h1 G((yg[g] - y_i)/h2) / sum_i K_h1,
 * G the y kernel's CDF: Phi for the Gaussian, (2 + 3t - t^3)/4 on [-1, 1] for
 * the Epanechnikov kernel.  Gaussian x weights are exp(e_i - max e) (FP64).
 * An Epanechnikov query with no x-neighbour inside h1 gets mean = NaN (0/0),
 * fat = 0 and F = NaN. */
typedef struct {
    const double *x, *y, *xq, *yq, *yg;
    int64_t N, Q;
    int d, G, kernel;
    double h1, h2;
    double *mean, *fat, *F;
    int64_t next;
    pthread_mutex_t mu;
} prod_job_t;

static double kernel_cdf(int kernel, double t) {
    if (kernel == 1) {
        if (t <= -1.0) return 0.0;
        if (t >= 1.0) return 1.0;
        return (2.0 + 3.0 * t - t * t * t) / 4.0;
    }
    return 0.5 * erfc(-t / sqrt(2.0));
}

static double kernel_pdf_y(int kernel, double t, double h2) {
    if (kernel == 1) return 0.75 * epan_prof(t * t, 1.0) / h2;
    return exp(-0.5 * t * t - LN_SQRT_2PI) / h2;
}

static void *prod_worker(void *arg) {
    prod_job_t *J = (prod_job_t *)arg;
    double *wx = malloc(sizeof(double) * J->N);
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t q = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (q >= J->Q) break;
        double m = -INFINITY;
        for (int64_t i = 0; i < J->N; ++i) {
            const double r2 = sqdist(J->xq + q * J->d, J->x + i * J->d, J->d);
            if (J->kernel == 1) {
                wx[i] = epan_prof(r2, J->h1);
            } else {
                wx[i] = -r2 / (2.0 * J->h1 * J->h1);
                if (wx[i] > m) m = wx[i];
            }
        }
        if (J->kernel != 1)
            for (int64_t i = 0; i < J->N; ++i) wx[i] = exp(wx[i] - m);
        double B = 0.0, S1 = 0.0;
        for (int64_t i = 0; i < J->N; ++i) {
            B += wx[i];
            S1 += wx[i] * J->y[i];
        }
        if (J->mean) J->mean[q] = S1 / B;
        if (J->fat) {
            double A = 0.0;
            for (int64_t i = 0; i < J->N; ++i)
                A += wx[i] * kernel_pdf_y(J->kernel, (J->yq[q] - J->y[i]) / J->h2, J->h2);
            J->fat[q] = B > 0.0 ? A / B : 0.0;
        }
        if (J->F)
            for (int g = 0; g < J->G; ++g) {
                double A = 0.0;
                for (int64_t i = 0; i < J->N; ++i)
                    A += wx[i] * kernel_cdf(J->kernel, (J->yg[g] - J->y[i]) / J->h2);
                J->F[q * J->G + g] = A / B;
            }
    }
    free(wx);
    return NULL;
}

/* mean[Q], fat[Q] (needs yq) and F[Q][G] (needs yg); any output may be NULL. */
void oracle_cond_products(const double *x, const double *y, int64_t N, int d, double h1, double h2,
                          const double *xq, const double *yq, int64_t Q, const double *yg, int G,
                          double *mean, double *fat, double *F, int n_threads, int kernel) {
    prod_job_t J;
    memset(&J, 0, sizeof(J));
    J.x = x; J.y = y; J.xq = xq; J.yq = yq; J.yg = yg; J.N = N; J.Q = Q; J.d = d; J.G = G;
    J.kernel = kernel; J.h1 = h1; J.h2 = h2; J.mean = mean; J.fat = fat; J.F = F;
    pthread_mutex_init(&J.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = malloc(sizeof(pthread_t) * n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, prod_worker, &J);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
}
