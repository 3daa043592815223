// One-dimensional grids in FP64 (Algorithm "VUP - Single probability" with
// the densities of Eq. VUP, every step in double precision).  One CTA per
// density: the pdf is evaluated at every midpoint and normalised, raw moments
// and central moments (second pass about the mean) are reduced with a fixed
// tree, and the histogram walks the bin-sorted points (the CSR form of the
// one-hot model matrix, Eq. MUP) one warp per bin.
#include "vup_internal.cuh"

#include <math.h>

namespace {

constexpr int kThreads = 256;

struct P1 {
    const uint8_t *kind;
    const double *mu, *sigma, *lo, *hi;
};

// Unnormalised density at midpoint a; Gaussian values are scaled by their
// value at the midpoint nearest the mean (removed by the normalisation).
__device__ __forceinline__ double g1(int kind, int64_t a, double lo, double h, double mu, double sg, double tlo,
                                     double thi, double u0sq, double &u) {
    const double x = __dadd_rn(lo, __dmul_rn((double)a + 0.5, h));
    u = (x - mu) / sg;
    if (kind == VUP_UNIFORM) {
        u = 0.0;
        const double half = __dmul_rn(0.5, sg);
        return fabs(__dsub_rn(x, mu)) <= half ? 1.0 : 0.0;
    }
    if (kind == VUP_TRUNCNORM && !(tlo <= x && x <= thi)) return 0.0;
    return exp(-0.5 * (u * u - u0sq));
}

__device__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

struct Geo1 {
    int64_t n;
    double lo, h;
};

__device__ __forceinline__ double u0sq_of(int kind, const Geo1 &G, double mu, double sg) {
    if (kind == VUP_UNIFORM) return 0.0;
    double c = (mu - G.lo) / G.h - 0.5;
    double an = fmin(fmax(floor(c + 0.5), 0.0), (double)(G.n - 1));
    double x = __dadd_rn(G.lo, __dmul_rn(an + 0.5, G.h));
    double u = (x - mu) / sg;
    return u * u;
}

template <bool kIpsa>
__global__ void __launch_bounds__(kThreads) k_1d(P1 p, Geo1 G, const double *__restrict__ y,
                                                 const int32_t *__restrict__ perm,
                                                 const int32_t *__restrict__ offsets, int B, int J,
                                                 double *__restrict__ raw, double *__restrict__ central,
                                                 float *__restrict__ hist, const double *__restrict__ grad,
                                                 float *__restrict__ dmu, float *__restrict__ dsg,
                                                 int *__restrict__ dstatus) {
    __shared__ double red[33];
    const int64_t k = blockIdx.x;
    const int kind = p.kind[k];
    const double mu = p.mu[k], sg = p.sigma[k];
    const double tlo = p.lo ? p.lo[k] : 0.0, thi = p.hi ? p.hi[k] : 0.0;
    const double u0sq = u0sq_of(kind, G, mu, sg);
    double z = 0.0, su = 0.0, su2 = 0.0, m[4] = {0, 0, 0, 0}, mu1[4] = {0, 0, 0, 0}, mu2[4] = {0, 0, 0, 0};
    for (int64_t a = threadIdx.x; a < G.n; a += blockDim.x) {
        double u;
        const double g = g1(kind, a, G.lo, G.h, mu, sg, tlo, thi, u0sq, u);
        const double yv = y[a];
        z += g;
        su += g * u;
        su2 += g * u * u;
        double pw = yv;
        for (int j = 0; j < 4; ++j) {
            m[j] += g * pw;
            if (kIpsa) {
                mu1[j] += g * u * pw;
                mu2[j] += g * u * u * pw;
            }
            pw *= yv;
        }
    }
    const double Z = block_sum(z, red);
    if (!(Z > 0.0)) {
        if (threadIdx.x == 0) atomicCAS(dstatus, 0, VUP_DSTAT_EMPTY);
        return;
    }
    double M[4];
    for (int j = 0; j < 4; ++j) M[j] = block_sum(m[j], red) / Z;
    if (kIpsa) {
        const double Eu = block_sum(su, red) / Z, Eu2 = block_sum(su2, red) / Z;
        const bool diff = kind != VUP_UNIFORM;
        double gm = 0.0, gs = 0.0;
        for (int j = 0; j < J; ++j) {
            const double S1 = block_sum(mu1[j], red) / Z, S2 = block_sum(mu2[j], red) / Z;
            const double dm = diff ? (S1 - Eu * M[j]) / sg : 0.0;
            const double ds = diff ? (S2 - Eu2 * M[j]) / sg : 0.0;
            if (grad) {
                gm += grad[k * J + j] * dm;
                gs += grad[k * J + j] * ds;
            } else if (threadIdx.x == 0) {
                dmu[k * J + j] = (float)dm;
                dsg[k * J + j] = (float)ds;
            }
        }
        if (grad && threadIdx.x == 0) {
            dmu[k] = (float)gm;
            dsg[k] = (float)gs;
        }
        return;
    }
    if (raw && threadIdx.x == 0)
        for (int j = 0; j < J; ++j) raw[k * J + j] = M[j];
    if (central) {
        const double mean = M[0];
        double c[4] = {0, 0, 0, 0};
        for (int64_t a = threadIdx.x; a < G.n; a += blockDim.x) {
            double u;
            const double g = g1(kind, a, G.lo, G.h, mu, sg, tlo, thi, u0sq, u);
            const double dv = y[a] - mean;
            double pw = dv;
            for (int j = 0; j < 4; ++j) {
                c[j] += g * pw;
                pw *= dv;
            }
        }
        double C[4];
        for (int j = 0; j < 4; ++j) C[j] = block_sum(c[j], red) / Z;
        if (threadIdx.x == 0) {
            central[k * J + 0] = mean;
            for (int j = 1; j < J; ++j) central[k * J + j] = C[j];
        }
    }
    if (hist) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int b = warp; b < B; b += nw) {
            double s = 0.0;
            for (int32_t t = offsets[b] + lane; t < offsets[b + 1]; t += 32) {
                double u;
                s += g1(kind, perm[t], G.lo, G.h, mu, sg, tlo, thi, u0sq, u);
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) hist[k * B + b] = (float)(s / Z);
        }
    }
}

}  // namespace

vup_status vup_propagate_1d(vup_grid g, const vup_densities *d, double *raw, double *central, float *hist,
                            cudaStream_t s) {
    P1 p{d->kind, d->mu, d->sigma, d->lo, d->hi};
    Geo1 G{g->n[0], g->lo[0], (g->hi[0] - g->lo[0]) / (double)g->n[0]};
    VUP_PROF("vup_1d_fp64", s, 1);
    k_1d<false><<<(unsigned)d->K, kThreads, 0, s>>>(p, G, g->y, g->perm, g->offsets, g->B, g->J, raw, central,
                                                    hist, nullptr, nullptr, nullptr, g->dstatus);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}

vup_status vup_ipsa_1d(vup_grid g, const vup_densities *d, const double *grad, float *dmu, float *dsg,
                       cudaStream_t s) {
    P1 p{d->kind, d->mu, d->sigma, d->lo, d->hi};
    Geo1 G{g->n[0], g->lo[0], (g->hi[0] - g->lo[0]) / (double)g->n[0]};
    VUP_PROF("ipsa_1d_fp64", s, 1);
    k_1d<true><<<(unsigned)d->K, kThreads, 0, s>>>(p, G, g->y, g->perm, g->offsets, g->B, g->J, nullptr, nullptr,
                                                   nullptr, grad, dmu, dsg, g->dstatus);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}
