/*
 * Host sanitizer run of the FP64 oracle (test infrastructure): compiled
 * together with oracle/vup_oracle.c under -fsanitize=address,undefined by
 * tests/test_oracle_sanitizers.py, it calls every oracle entry point on small
 * ragged 1-D, 2-D and 3-D grids with every density kind and model, so that an
 * out-of-bounds index, a leak or undefined arithmetic in the oracle stops the
 * run.  It also checks the invariants sum_b H = 1 and M_0 = 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

double oracle_grid_coord(double lo, double hi, int64_t n, int64_t a);
int oracle_eval_model(int model_id, const double *theta, int ndim, const int64_t *n, const double *lo,
                      const double *hi, double *y);
void oracle_bins(int64_t N, const double *y, int B, int32_t *bins, double *ymin_out, double *ymax_out);
int oracle_weights(int ndim, const int64_t *n, const double *lo, const double *hi, int64_t K, const uint8_t *kind,
                   const double *mu, const double *sigma, const double *tlo, const double *thi, int64_t k,
                   double *W, double *Z_out);
int oracle_propagate(int ndim, const int64_t *n, const double *lo, const double *hi, const double *y,
                     const int32_t *bins, int B, int J, int64_t n_sel, const int64_t *k_sel, int64_t K,
                     const uint8_t *kind, const double *mu, const double *sigma, const double *tlo,
                     const double *thi, double *raw, double *central, double *hist, double *wsum, int nthreads);
int oracle_ipsa(int ndim, const int64_t *n, const double *lo, const double *hi, const double *y, int J,
                int64_t n_sel, const int64_t *k_sel, int64_t K, const uint8_t *kind, const double *mu,
                const double *sigma, const double *tlo, const double *thi, double *dmu, double *dsigma,
                int nthreads);
int oracle_ipsa_scale(int ndim, const int64_t *n, const double *lo, const double *hi, const double *y, int J,
                      int64_t n_sel, const int64_t *k_sel, int64_t K, const uint8_t *kind, const double *mu,
                      const double *sigma, const double *tlo, const double *thi, double *cmu, double *csg,
                      int nthreads);
int oracle_model_at(int model_id, const double *theta, int ndim, int64_t K, const double *x, double *y);
int oracle_deviation_moments(int ndim, const int64_t *n, const double *lo, const double *hi, const double *y,
                             int J, int64_t S, const int64_t *rows, const double *yref, int64_t K,
                             const uint8_t *kind, const double *mu, const double *sigma, const double *tlo,
                             const double *thi, double *out);
void oracle_ipsa_matrix(int64_t K, int B, double ymin, double ymax, const double *H, const double *yref, int nd,
                        double dlo, double dhi, double *out);
void oracle_sa_fields(int64_t K, int nb, const double *H, double level, const double *rho, int32_t *argmax,
                      int32_t *ci, double *global);
int oracle_posterior_means(int ndim, const int64_t *n, const double *lo, const double *hi, const int32_t *bins,
                           int B, int64_t S, const int64_t *rows, int64_t K, const uint8_t *kind,
                           const double *mu, const double *sigma, const double *tlo, const double *thi,
                           double *post);

static int fails = 0;
#define CHECK(c, ...)                          \
    do {                                       \
        if (!(c)) {                            \
            fprintf(stderr, __VA_ARGS__);      \
            fprintf(stderr, "\n");             \
            ++fails;                           \
        }                                      \
    } while (0)

/* deterministic uniform numbers in [0, 1) (a 64-bit LCG; inputs only) */
static uint64_t lcg = 88172645463325252ull;
static double urand(void) {
    lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(lcg >> 11) * (1.0 / 9007199254740992.0);
}

static void run_case(int ndim, const int64_t *n, int model, const double *theta, int B, int64_t K) {
    const int J = 4;
    double lo[3], hi[3];
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) {
        lo[d] = -1.0 - urand();
        hi[d] = 1.0 + urand();
        N *= n[d];
    }
    if (model == 4) { /* the oscillator's domain: omega in [0.5, 5], damping in [0.01, 0.9] */
        lo[0] = 0.5, hi[0] = 5.0;
        lo[1] = 0.01, hi[1] = 0.9;
    }
    double *y = malloc(sizeof(double) * N);
    int32_t *bins = malloc(sizeof(int32_t) * N);
    uint8_t *kind = malloc((size_t)K * ndim);
    double *mu = malloc(sizeof(double) * K * ndim), *sg = malloc(sizeof(double) * K * ndim);
    double *tl = malloc(sizeof(double) * K * ndim), *th = malloc(sizeof(double) * K * ndim);
    for (int64_t p = 0; p < K * ndim; ++p) {
        const int d = (int)(p % ndim);
        const double w = hi[d] - lo[d];
        kind[p] = (uint8_t)(p % 3);
        mu[p] = lo[d] + (0.2 + 0.6 * urand()) * w;
        sg[p] = (kind[p] == 1 ? 0.3 + 0.5 * urand() : 0.1 + 0.3 * urand()) * w;
        tl[p] = mu[p] - 0.25 * w;
        th[p] = mu[p] + 0.3 * w;
    }
    CHECK(oracle_eval_model(model, theta, ndim, n, lo, hi, y) == 0, "eval_model %d", model);
    double ymin, ymax;
    oracle_bins(N, y, B, bins, &ymin, &ymax);
    int64_t *rows = malloc(sizeof(int64_t) * K);
    for (int64_t k = 0; k < K; ++k) rows[k] = K - 1 - k;
    double *W = malloc(sizeof(double) * N), Z;
    CHECK(oracle_weights(ndim, n, lo, hi, K, kind, mu, sg, tl, th, K - 1, W, &Z) == 0, "weights");
    double *raw = malloc(sizeof(double) * K * J), *cen = malloc(sizeof(double) * K * J);
    double *hist = malloc(sizeof(double) * K * B), *ws = malloc(sizeof(double) * K);
    CHECK(oracle_propagate(ndim, n, lo, hi, y, bins, B, J, K, rows, K, kind, mu, sg, tl, th, raw, cen, hist, ws,
                           1) == 0,
          "propagate");
    for (int64_t s = 0; s < K; ++s) {
        double h = 0.0;
        for (int b = 0; b < B; ++b) h += hist[s * B + b];
        CHECK(fabs(h - 1.0) < 1e-12 && fabs(ws[s] - 1.0) < 1e-12, "sum H %g, M0 %g", h, ws[s]);
    }
    double *dmu = malloc(sizeof(double) * K * ndim * J), *dsg = malloc(sizeof(double) * K * ndim * J);
    double *cmu = malloc(sizeof(double) * K * ndim * J), *csg = malloc(sizeof(double) * K * ndim * J);
    CHECK(oracle_ipsa(ndim, n, lo, hi, y, J, K, rows, K, kind, mu, sg, tl, th, dmu, dsg, 1) == 0, "ipsa");
    CHECK(oracle_ipsa_scale(ndim, n, lo, hi, y, J, K, rows, K, kind, mu, sg, tl, th, cmu, csg, 1) == 0,
          "ipsa_scale");
    for (int64_t e = 0; e < K * ndim * J; ++e)
        CHECK(fabs(dmu[e]) <= cmu[e] * (1 + 1e-12) + 1e-300 && fabs(dsg[e]) <= csg[e] * (1 + 1e-12) + 1e-300,
              "ipsa bound");
    double *yref = malloc(sizeof(double) * K);
    CHECK(oracle_model_at(model, theta, ndim, K, mu, yref) == 0, "model_at");
    double *dev = malloc(sizeof(double) * K * J);
    CHECK(oracle_deviation_moments(ndim, n, lo, hi, y, J, K, rows, yref, K, kind, mu, sg, tl, th, dev) == 0,
          "deviation moments");
    const int nd = 2 * B + 1;
    double *ipm = malloc(sizeof(double) * K * nd);
    oracle_ipsa_matrix(K, B, ymin, ymax, hist, yref, nd, -(ymax - ymin), ymax - ymin, ipm);
    double *rho = malloc(sizeof(double) * K), *glob = malloc(sizeof(double) * B);
    for (int64_t k = 0; k < K; ++k) rho[k] = 1.0 + (double)k;
    int32_t *amax = malloc(sizeof(int32_t) * K), *ci = malloc(sizeof(int32_t) * 2 * K);
    oracle_sa_fields(K, B, hist, 0.9, rho, amax, ci, glob);
    for (int64_t k = 0; k < K; ++k) CHECK(amax[k] >= 0 && amax[k] < B && ci[2 * k] <= ci[2 * k + 1], "fields");
    if (ndim >= 2) {
        double *post = malloc(sizeof(double) * K * B * ndim);
        CHECK(oracle_posterior_means(ndim, n, lo, hi, bins, B, K, rows, K, kind, mu, sg, tl, th, post) == 0,
              "posterior means");
        free(post);
    }
    free(y); free(bins); free(kind); free(mu); free(sg); free(tl); free(th); free(rows); free(W);
    free(raw); free(cen); free(hist); free(ws); free(dmu); free(dsg); free(cmu); free(csg); free(yref);
    free(dev); free(ipm); free(rho); free(glob); free(amax); free(ci);
}

int main(void) {
    const double t1[2] = {1.0, 0.1}, t2[2] = {1.0, 7.0}, t3[2] = {7.0, 0.1}, t4[1] = {3.0};
    const double tp[7] = {0.5, 1.0, -0.3, 2.0, 0.1, -1.5, 0.7};
    const int64_t n1[1] = {37}, n2[2] = {13, 29}, n3[3] = {7, 11, 9}, n2b[2] = {31, 5};
    run_case(1, n1, 1, t1, 7, 5);
    run_case(1, n1, 6, tp, 1, 3);
    run_case(2, n2, 2, t2, 16, 6);
    run_case(2, n2b, 4, t4, 9, 4);
    run_case(2, n2, 5, NULL, 33, 5);
    run_case(2, n2, 6, tp, 2, 4);
    run_case(3, n3, 3, t3, 64, 5);
    run_case(3, n3, 6, tp, 5, 3);
    if (fails) {
        fprintf(stderr, "%d checks failed\n", fails);
        return 1;
    }
    printf("sanitized oracle run ok\n");
    return 0;
}
