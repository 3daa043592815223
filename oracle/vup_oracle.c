/*
 * FP64 CPU oracle for Vectorized Uncertainty Propagation (VUP).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA path.
 *
 * Every quantity is computed from its plain definition with straightforward
 * loops over every grid point, in IEEE double precision, in the order the
 * paper states the method:
 *
 *   1. a uniform grid of midpoints (Sec. 3, composite midpoint rule;
 *      Algorithm "VUP - Single probability", first step);
 *   2. the model evaluated once per grid point (Eq. modelfunction, Sec. 2);
 *   3. the input pdf evaluated at every grid point and normalised over the
 *      grid (Algorithm "VUP - Single probability"; Sec. 5.3 hard truncation
 *      at the domain boundary followed by renormalisation);
 *   4. the output probabilities of Eq. 4 / Eq. 5: every grid point's input
 *      probability is summed into the output bin its model value falls in
 *      (the one-hot model matrix of Eq. MUP applied to each column of the
 *      input probability matrix, Eq. VUP);
 *   5. raw moments sum_i W[k,i] y_i^j and central moments about the mean,
 *      the expectation fields read off the output probability matrix
 *      (Sec. 5.2 coarse-grained quantities; Fig. 4c);
 *   6. IPSA sensitivities of those moments to the input uncertainty
 *      parameters, from differentiating W = g / sum(g) exactly.
 *
 * The weights are NOT factored per axis: the product density is evaluated
 * at each tensor-grid point and normalised by its sum over all N points.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_GAUSS 0
#define OR_UNIFORM 1
#define OR_TRUNCNORM 2

/* Midpoint x_{d,a} = lo + (a + 1/2) h with h = (hi - lo) / n (Sec. 3). */
double oracle_grid_coord(double lo, double hi, int64_t n, int64_t a)
{
    double h = (hi - lo) / (double)n;
    double t = (double)a + 0.5;
    double off = t * h;
    return lo + off;
}

/* Split flat row-major index i into per-axis indices (axis 0 slowest). */
static void unflatten(int ndim, const int64_t *n, int64_t i, int64_t *a)
{
    for (int d = ndim - 1; d >= 0; --d) {
        a[d] = i % n[d];
        i /= n[d];
    }
}

/*
 * Built-in models (Sec. 2, M(x, alpha) = y; Sec. 4.1 timing model;
 * Sec. 5.3 IPSA example).  Operation order is fixed so a reader can
 * reproduce every rounding.
 */
static double model_value(int model_id, const double *th, int ndim, const double *x)
{
    switch (model_id) {
    case 1: { /* th0 sin x + th1 x^2 */
        double s = sin(x[0]);
        double q = x[0] * x[0];
        double a = th[0] * s;
        double b = th[1] * q;
        return a + b;
    }
    case 2: { /* th0 sin x1 + th1 sin^2 x2   (Sec. 4.1 model) */
        double s1 = sin(x[0]);
        double s2 = sin(x[1]);
        double q = s2 * s2;
        double a = th[0] * s1;
        double b = th[1] * q;
        return a + b;
    }
    case 3: { /* sin x1 + th0 sin^2 x2 + th1 x3^4 sin x1 */
        double s1 = sin(x[0]);
        double s2 = sin(x[1]);
        double q = s2 * s2;
        double x2 = x[2] * x[2];
        double x4 = x2 * x2;
        double b = th[0] * q;
        double c = th[1] * x4;
        double c2 = c * s1;
        double r = s1 + b;
        return r + c2;
    }
    case 4: { /* damped oscillator, x = (omega, zeta), th0 = T */
        double w = x[0], z = x[1], T = th[0];
        double zw = z * w;
        double e = exp(-(zw * T));
        double om = 1.0 - z * z;
        double wd = w * sqrt(om);
        double c = cos(wd * T);
        return e * c;
    }
    case 5: { /* x^2 + 5 sin(3x) + alpha   (Sec. 5.3 example) */
        double q = x[0] * x[0];
        double t = 3.0 * x[0];
        double s = 5.0 * sin(t);
        double r = q + s;
        return r + x[1];
    }
    case 6: { /* th0 + sum_d (th[1+2d] x_d + th[2+2d] x_d^2) */
        double r = th[0];
        for (int d = 0; d < ndim; ++d) {
            double a = th[1 + 2 * d] * x[d];
            double q = x[d] * x[d];
            double b = th[2 + 2 * d] * q;
            r = r + a;
            r = r + b;
        }
        return r;
    }
    default:
        return NAN;
    }
}

static int model_ndim_ok(int model_id, int ndim)
{
    switch (model_id) {
    case 1: return ndim == 1;
    case 2: case 4: case 5: return ndim == 2;
    case 3: return ndim == 3;
    case 6: return ndim >= 1 && ndim <= 3;
    default: return 0;
    }
}

/* y_i = M(x_i; theta) for every point of the tensor grid (Algorithm
 * "VUP - Single probability", second step).  Returns 0 on success. */
int oracle_eval_model(int model_id, const double *theta, int ndim, const int64_t *n,
                      const double *lo, const double *hi, double *y)
{
    if (!model_ndim_ok(model_id, ndim)) return 1;
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    for (int64_t i = 0; i < N; ++i) {
        int64_t a[3];
        double x[3];
        unflatten(ndim, n, i, a);
        for (int d = 0; d < ndim; ++d) x[d] = oracle_grid_coord(lo[d], hi[d], n[d], a[d]);
        y[i] = model_value(model_id, theta, ndim, x);
    }
    return 0;
}

/*
 * Output bins of Eq. 4: B bins of equal width over [min y, max y],
 * half-open [e_b, e_{b+1}) with the last bin closed:
 *   t = (y - ymin) / (ymax - ymin),  bin = min(floor(t * B), B - 1).
 * A constant model (ymax == ymin) puts every point in bin 0.
 */
void oracle_bins(int64_t N, const double *y, int B, int32_t *bins, double *ymin_out,
                 double *ymax_out)
{
    double ymin = y[0], ymax = y[0];
    for (int64_t i = 1; i < N; ++i) {
        if (y[i] < ymin) ymin = y[i];
        if (y[i] > ymax) ymax = y[i];
    }
    double range = ymax - ymin;
    for (int64_t i = 0; i < N; ++i) {
        int32_t b = 0;
        if (range > 0.0) {
            double t = (y[i] - ymin) / range;
            double tb = t * (double)B;
            double f = floor(tb);
            b = (int32_t)f;
            if (b > B - 1) b = B - 1;
            if (b < 0) b = 0;
        }
        bins[i] = b;
    }
    *ymin_out = ymin;
    *ymax_out = ymax;
}

/*
 * One axis of the input density at coordinate x (Eq. gaussh; uniform and
 * truncated normal as the other measurement-uncertainty shapes named in
 * Sec. 5.2).  Unnormalised: the grid normalisation divides it out.
 */
static double density_1d(int kind, double x, double mu, double sigma, double tlo, double thi)
{
    if (kind == OR_UNIFORM) {
        double half = 0.5 * sigma;
        double dx = fabs(x - mu);
        return dx <= half ? 1.0 : 0.0;
    }
    if (kind == OR_TRUNCNORM) {
        if (!(tlo <= x && x <= thi)) return 0.0;
    }
    double u = x - mu;
    double s2 = sigma * sigma;
    double e = (u * u) / (2.0 * s2);
    return exp(-e);
}

typedef struct {
    int ndim;
    const int64_t *n;
    const double *lo, *hi;
    int64_t K;
    const uint8_t *kind;
    const double *mu, *sigma, *tlo, *thi;
} oracle_dens;

/* g_k(x_i) = prod_d rho_{k,d}(x_{d,a_d}) at every grid point. */
static void eval_g(const oracle_dens *D, int64_t k, int64_t N, double *g)
{
    int nd = D->ndim;
    for (int64_t i = 0; i < N; ++i) {
        int64_t a[3];
        unflatten(nd, D->n, i, a);
        double v = 1.0;
        for (int d = 0; d < nd; ++d) {
            double x = oracle_grid_coord(D->lo[d], D->hi[d], D->n[d], a[d]);
            int64_t p = k * nd + d;
            v = v * density_1d(D->kind[p], x, D->mu[p], D->sigma[p], D->tlo[p], D->thi[p]);
        }
        g[i] = v;
    }
}

/*
 * Normalised input probability vector W[k, :] = g / sum_i g (Algorithm
 * "VUP - Single probability": evaluate the pdf on the grid and normalise;
 * Sec. 5.3: truncate at the domain and renormalise).  Returns the sum of g
 * (0 means the support holds no grid point).
 */
static double weights(const oracle_dens *D, int64_t k, int64_t N, double *W)
{
    eval_g(D, k, N, W);
    double Z = 0.0;
    for (int64_t i = 0; i < N; ++i) Z += W[i];
    if (Z > 0.0)
        for (int64_t i = 0; i < N; ++i) W[i] = W[i] / Z;
    return Z;
}

int oracle_weights(int ndim, const int64_t *n, const double *lo, const double *hi, int64_t K,
                   const uint8_t *kind, const double *mu, const double *sigma, const double *tlo,
                   const double *thi, int64_t k, double *W, double *Z_out)
{
    oracle_dens D = {ndim, n, lo, hi, K, kind, mu, sigma, tlo, thi};
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    double Z = weights(&D, k, N, W);
    if (Z_out) *Z_out = Z;
    return Z > 0.0 ? 0 : 5;
}

/*
 * VUP forward pass for a selection of distributions k (Eq. VUP applied
 * column by column):
 *   raw[s][j-1]     = sum_i W[k,i] y_i^j                         (j = 1..J)
 *   central[s][0]   = raw[s][0]  (the mean)
 *   central[s][j-1] = sum_i W[k,i] (y_i - mean)^j                (j = 2..J)
 *   hist[s][b]      = sum_i W[k,i] [bins_i == b]                 (Eq. 4/5)
 *   wsum[s]         = sum_i W[k,i]
 * Any output pointer may be NULL.  Returns 0, or 5 if some selected
 * distribution has no grid point in its support.
 */
int oracle_propagate(int ndim, const int64_t *n, const double *lo, const double *hi,
                     const double *y, const int32_t *bins, int B, int J, int64_t n_sel,
                     const int64_t *k_sel, int64_t K, const uint8_t *kind, const double *mu,
                     const double *sigma, const double *tlo, const double *thi, double *raw,
                     double *central, double *hist, double *wsum, int nthreads)
{
    oracle_dens D = {ndim, n, lo, hi, K, kind, mu, sigma, tlo, thi};
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *W = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < n_sel; ++s) {
            int64_t k = k_sel[s];
            double Z = weights(&D, k, N, W);
            if (!(Z > 0.0)) {
#pragma omp atomic write
                status = 5;
                continue;
            }
            if (wsum) {
                double t = 0.0;
                for (int64_t i = 0; i < N; ++i) t += W[i];
                wsum[s] = t;
            }
            double m1 = 0.0;
            for (int j = 1; j <= J; ++j) {
                double acc = 0.0;
                for (int64_t i = 0; i < N; ++i) {
                    double p = 1.0;
                    for (int e = 0; e < j; ++e) p = p * y[i];
                    acc += W[i] * p;
                }
                if (raw) raw[s * J + (j - 1)] = acc;
                if (j == 1) m1 = acc;
            }
            if (central) {
                central[s * J + 0] = m1;
                for (int j = 2; j <= J; ++j) {
                    double acc = 0.0;
                    for (int64_t i = 0; i < N; ++i) {
                        double dv = y[i] - m1;
                        double p = 1.0;
                        for (int e = 0; e < j; ++e) p = p * dv;
                        acc += W[i] * p;
                    }
                    central[s * J + (j - 1)] = acc;
                }
            }
            if (hist && bins) {
                double *h = hist + s * (int64_t)B;
                for (int b = 0; b < B; ++b) h[b] = 0.0;
                for (int64_t i = 0; i < N; ++i) h[bins[i]] += W[i];
            }
        }
        free(W);
    }
    return status;
}

/*
 * IPSA sensitivities of the raw moments to the input-uncertainty
 * parameters (the derivative of each output statistic with respect to the
 * measurement uncertainty at location k; Sec. 5.2, Eq. IPSAvar family).
 * With W = g / sum(g) and g a product of per-axis densities,
 *   dW/dp = W (s_p - sum_i W s_p),   s_p = d log g / dp,
 * so   dM_j/dp = sum_i W_i (s_p(i) - sbar_p) y_i^j.
 * Gaussian and truncated-normal axes (bounds held fixed):
 *   s_mu = (x - mu) / sigma^2,   s_sigma = (x - mu)^2 / sigma^3.
 * Uniform axes have non-differentiable support edges; their entries are 0.
 * Outputs dmu, dsigma: [n_sel][ndim][J].
 */
int oracle_ipsa(int ndim, const int64_t *n, const double *lo, const double *hi, const double *y,
                int J, int64_t n_sel, const int64_t *k_sel, int64_t K, const uint8_t *kind,
                const double *mu, const double *sigma, const double *tlo, const double *thi,
                double *dmu, double *dsigma, int nthreads)
{
    oracle_dens D = {ndim, n, lo, hi, K, kind, mu, sigma, tlo, thi};
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *W = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < n_sel; ++s) {
            int64_t k = k_sel[s];
            double Z = weights(&D, k, N, W);
            if (!(Z > 0.0)) {
#pragma omp atomic write
                status = 5;
                continue;
            }
            for (int d = 0; d < ndim; ++d) {
                int64_t p = k * ndim + d;
                int differentiable = D.kind[p] != OR_UNIFORM;
                double m = mu[p], sg = sigma[p];
                double sbar_mu = 0.0, sbar_sg = 0.0;
                for (int64_t i = 0; i < N; ++i) {
                    int64_t a[3];
                    unflatten(ndim, n, i, a);
                    double x = oracle_grid_coord(lo[d], hi[d], n[d], a[d]);
                    double u = x - m;
                    double smu = u / (sg * sg);
                    double ssg = (u * u) / (sg * sg * sg);
                    sbar_mu += W[i] * smu;
                    sbar_sg += W[i] * ssg;
                }
                for (int j = 1; j <= J; ++j) {
                    double am = 0.0, as = 0.0;
                    for (int64_t i = 0; i < N; ++i) {
                        int64_t a[3];
                        unflatten(ndim, n, i, a);
                        double x = oracle_grid_coord(lo[d], hi[d], n[d], a[d]);
                        double u = x - m;
                        double smu = u / (sg * sg);
                        double ssg = (u * u) / (sg * sg * sg);
                        double pw = 1.0;
                        for (int e = 0; e < j; ++e) pw = pw * y[i];
                        am += W[i] * (smu - sbar_mu) * pw;
                        as += W[i] * (ssg - sbar_sg) * pw;
                    }
                    int64_t o = (s * ndim + d) * J + (j - 1);
                    dmu[o] = differentiable ? am : 0.0;
                    dsigma[o] = differentiable ? as : 0.0;
                }
            }
        }
        free(W);
    }
    return status;
}

/*
 * Condition scale of the IPSA sensitivities above (test infrastructure for
 * the tolerance of a reduced-precision computation of the same sums).  The
 * derivative is a covariance, dM_j/dp = sum_i W s_p y^j - sbar_p sum_i W y^j;
 * the sum of the absolute values of all of its products is
 *   cmu[s][d][j-1] = sum_i W |s_mu| |y|^j + |sbar_mu| sum_i W |y|^j,
 *   csg[s][d][j-1] = sum_i W  s_sg  |y|^j +  sbar_sg  sum_i W |y|^j,
 * the quantity a rounding error relative to each product is measured
 * against (as sum_i W |y|^j is for the raw moments).  Every axis gets its
 * scale, uniform ones included.  Outputs [n_sel][ndim][J].
 */
int oracle_ipsa_scale(int ndim, const int64_t *n, const double *lo, const double *hi, const double *y,
                      int J, int64_t n_sel, const int64_t *k_sel, int64_t K, const uint8_t *kind,
                      const double *mu, const double *sigma, const double *tlo, const double *thi,
                      double *cmu, double *csg, int nthreads)
{
    oracle_dens D = {ndim, n, lo, hi, K, kind, mu, sigma, tlo, thi};
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *W = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < n_sel; ++s) {
            int64_t k = k_sel[s];
            double Z = weights(&D, k, N, W);
            if (!(Z > 0.0)) {
#pragma omp atomic write
                status = 5;
                continue;
            }
            for (int d = 0; d < ndim; ++d) {
                int64_t p = k * ndim + d;
                double m = mu[p], sg = sigma[p];
                double sbar_mu = 0.0, sbar_sg = 0.0;
                for (int64_t i = 0; i < N; ++i) {
                    int64_t a[3];
                    unflatten(ndim, n, i, a);
                    double x = oracle_grid_coord(lo[d], hi[d], n[d], a[d]);
                    double u = x - m;
                    sbar_mu += W[i] * (u / (sg * sg));
                    sbar_sg += W[i] * ((u * u) / (sg * sg * sg));
                }
                for (int j = 1; j <= J; ++j) {
                    double am = 0.0, as = 0.0, ay = 0.0;
                    for (int64_t i = 0; i < N; ++i) {
                        int64_t a[3];
                        unflatten(ndim, n, i, a);
                        double x = oracle_grid_coord(lo[d], hi[d], n[d], a[d]);
                        double u = x - m;
                        double smu = u / (sg * sg);
                        double ssg = (u * u) / (sg * sg * sg);
                        double pw = 1.0;
                        for (int e = 0; e < j; ++e) pw = pw * fabs(y[i]);
                        am += W[i] * fabs(smu) * pw;
                        as += W[i] * ssg * pw;
                        ay += W[i] * pw;
                    }
                    int64_t o = (s * ndim + d) * J + (j - 1);
                    cmu[o] = am + fabs(sbar_mu) * ay;
                    csg[o] = as + sbar_sg * ay;
                }
            }
        }
        free(W);
    }
    return status;
}

/* ------------------------------------------------------------------------
 * IPSA coarse-grained quantities (Sec. 5.2)
 * ---------------------------------------------------------------------- */

/* The model at arbitrary input points, e.g. the estimated values
 * y(l) = M(l, 0) at the densities' centres (Sec. 5.2: the deviations of
 * the IPSA probability matrix are measured from them).  x is [K][ndim]. */
int oracle_model_at(int model_id, const double *theta, int ndim, int64_t K, const double *x, double *y)
{
    if (!model_ndim_ok(model_id, ndim)) return 1;
    for (int64_t k = 0; k < K; ++k) y[k] = model_value(model_id, theta, ndim, x + k * ndim);
    return 0;
}

/* Deviation moments about the estimated values, from their definition:
 * out[s][j-1] = sum_i W[k,i] (y_i - yref[k])^j, j = 1..J, for the selected
 * rows k = rows[s].  j = 2 gives twice the local expected square deviation
 * Delta^2 of Eq. IPSAvar (the 1/2 of that equation is applied by callers). */
int oracle_deviation_moments(int ndim, const int64_t *n, const double *lo, const double *hi, const double *y,
                             int J, int64_t S, const int64_t *rows, const double *yref, int64_t K,
                             const uint8_t *kind, const double *mu, const double *sigma, const double *tlo,
                             const double *thi, double *out)
{
    oracle_dens D = {ndim, n, lo, hi, K, kind, mu, sigma, tlo, thi};
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    double *W = (double *)malloc(sizeof(double) * N);
    if (!W) return 2;
    int status = 0;
    for (int64_t s = 0; s < S; ++s) {
        int64_t k = rows[s];
        if (weights(&D, k, N, W) <= 0.0) {
            status = 1;
            continue;
        }
        for (int j = 1; j <= J; ++j) {
            double acc = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double u = y[i] - yref[k];
                double p = 1.0;
                for (int e = 0; e < j; ++e) p = p * u;
                acc += W[i] * p;
            }
            out[s * J + (j - 1)] = acc;
        }
    }
    free(W);
    return status;
}

/*
 * IPSA probability matrix (Eq. IPSA): every column of the output
 * probability matrix translated by -yref[k] (y -> dy = y - y(l)) and
 * collected on one grid of deviations: nd bins of width (dhi - dlo) / nd
 * starting at dlo.  Output bin b of [ymin, ymax] (B bins) stands for its
 * centre c_b = ymin + (b + 1/2) w; its mass goes to deviation bin
 * floor((c_b - yref[k] - dlo) / wd), clamped to [0, nd - 1] so that every
 * column keeps its mass.  Sums run over b in increasing order.
 */
void oracle_ipsa_matrix(int64_t K, int B, double ymin, double ymax, const double *H, const double *yref,
                        int nd, double dlo, double dhi, double *out)
{
    double w = (ymax - ymin) / (double)B;
    double wd = (dhi - dlo) / (double)nd;
    for (int64_t k = 0; k < K; ++k) {
        double *o = out + k * nd;
        for (int e = 0; e < nd; ++e) o[e] = 0.0;
        for (int b = 0; b < B; ++b) {
            double t = (double)b + 0.5;
            double c = ymin + t * w;
            double dy = c - yref[k];
            double f = floor((dy - dlo) / wd);
            int e = f < 0.0 ? 0 : (f > (double)(nd - 1) ? nd - 1 : (int)f);
            o[e] += H[k * B + b];
        }
    }
}

/*
 * Coarse-grained fields of one probability vector per row (Sec. 5.2: the
 * maximum probability per l and confidence intervals that vary with l),
 * and the global vector marginalised over l with weights rho (uniform when
 * rho is NULL):
 *   argmax[k] = the first bin of maximum probability;
 *   ci[k] = (lo, hi): lo the first bin whose cumulative mass exceeds
 *           (1 - level)/2 of the row total, hi the first bin whose
 *           cumulative mass reaches (1 + level)/2 of it.  The paper fixes
 *           no precision for these; they are taken in FP32 (the precision
 *           of the probabilities themselves): sums in bin order, each
 *           operation rounded to float;
 *   global[b] = sum_k rho_k H[k][b] / sum_k rho_k.
 */
void oracle_sa_fields(int64_t K, int nb, const double *H, double level, const double *rho, int32_t *argmax,
                      int32_t *ci, double *global)
{
    double lo_q = 0.5 * (1.0 - level), hi_q = 0.5 * (1.0 + level);
    for (int b = 0; b < nb; ++b) global[b] = 0.0;
    double rsum = 0.0;
    for (int64_t k = 0; k < K; ++k) {
        const double *h = H + k * nb;
        int am = 0;
        float total = 0.0f;
        for (int b = 0; b < nb; ++b) {
            if (h[b] > h[am]) am = b;
            total = total + (float)h[b];
        }
        argmax[k] = am;
        float tl = (float)lo_q * total, th = (float)hi_q * total;
        float cum = 0.0f;
        int lo = nb - 1, hi = nb - 1, have_lo = 0, have_hi = 0;
        for (int b = 0; b < nb; ++b) {
            cum = cum + (float)h[b];
            if (!have_lo && cum > tl) { lo = b; have_lo = 1; }
            if (!have_hi && cum >= th) { hi = b; have_hi = 1; }
        }
        ci[2 * k] = lo;
        ci[2 * k + 1] = hi;
        double r = rho ? rho[k] : 1.0;
        rsum += r;
        for (int b = 0; b < nb; ++b) global[b] += r * h[b];
    }
    if (rsum > 0.0)
        for (int b = 0; b < nb; ++b) global[b] = global[b] / rsum;
}

/*
 * Bayes-inverted model matrix applied to the input coordinates (Sec. 3, the
 * inverted model matrix M_{(x,a),y} built from Bayes' theorem): for row k
 * and output bin b, the posterior p(x_i | y in b, l_k) = W[k,i] [bin_i = b]
 * / H[k,b], and its mean per input axis,
 *   post[s][b][d] = sum_{i in b} W[k,i] x_{d,i} / H[k,b]
 * (0 for a bin of zero probability).  Also the identity of the footnote on
 * the inverted matrix, in its first-moment form: sum_b H[k,b] post[b][d]
 * equals the input mean sum_i W[k,i] x_{d,i}.
 */
int oracle_posterior_means(int ndim, const int64_t *n, const double *lo, const double *hi, const int32_t *bins,
                           int B, int64_t S, const int64_t *rows, int64_t K, const uint8_t *kind, const double *mu,
                           const double *sigma, const double *tlo, const double *thi, double *post)
{
    oracle_dens D = {ndim, n, lo, hi, K, kind, mu, sigma, tlo, thi};
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    double *W = (double *)malloc(sizeof(double) * N);
    double *h = (double *)malloc(sizeof(double) * B);
    if (!W || !h) {
        free(W);
        free(h);
        return 2;
    }
    int status = 0;
    for (int64_t s = 0; s < S; ++s) {
        int64_t k = rows[s];
        double *o = post + s * (int64_t)B * ndim;
        if (weights(&D, k, N, W) <= 0.0) {
            status = 1;
            continue;
        }
        for (int b = 0; b < B; ++b) h[b] = 0.0;
        for (int64_t e = 0; e < (int64_t)B * ndim; ++e) o[e] = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            int64_t a[3];
            unflatten(ndim, n, i, a);
            h[bins[i]] += W[i];
            for (int d = 0; d < ndim; ++d)
                o[(int64_t)bins[i] * ndim + d] += W[i] * oracle_grid_coord(lo[d], hi[d], n[d], a[d]);
        }
        for (int b = 0; b < B; ++b)
            for (int d = 0; d < ndim; ++d)
                o[(int64_t)b * ndim + d] = h[b] > 0.0 ? o[(int64_t)b * ndim + d] / h[b] : 0.0;
    }
    free(W);
    free(h);
    return status;
}
