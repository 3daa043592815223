// Density preparation: the input pdfs evaluated on the grid and normalised
// (Algorithm "VUP - Single probability": evaluate the input pdf at the grid
// points and normalise; Sec. 5.3: hard truncation at the domain boundary and
// renormalisation; Eq. gaussh Gaussian measurement uncertainty).
//
// Product densities factor over axes, so W[k, i] = prod_d g_d(k, a_d) / Z_d(k)
// with Z_d = sum_a g_d(k, a).  This kernel writes the per-axis factor tables
// g_d[a][k] (K x sum_d n_d floats -- never the K x N weights) and the FP64
// normalisation statistics.  The contraction and histogram kernels form W on
// the fly as products of these factors.
#include "vup_internal.cuh"

#include <math.h>

#include <algorithm>

namespace {

struct DensIn {
    const uint8_t *kind;
    const double *mu, *sigma, *lo, *hi;
};

// Neumaier-compensated FP32 accumulator.
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        float t = s + v;
        if (fabsf(s) >= fabsf(v)) c += (s - t) + v; else c += (v - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Error-free FP32 transformations (Knuth two-sum, FMA two-product).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Constants of one (k, d) Gaussian factor in index space, as FP32 pairs.
struct GaussArg {
    double nk;       // integer part of the mean's index coordinate
    float fh, fl;    // fractional part f = fh + fl
    float rh, rl;    // r = h / sigma = rh + rl
    float qh, ql;    // u0^2 = qh + ql (u at the midpoint nearest the mean)
};

// Per-axis density value at midpoint a (unnormalised), and u = ((a - n) - f) r.
// The exponent 0.5 (u^2 - u0^2) is carried as an FP32 pair (error ~2^-44
// relative) and exp is split, exp(-(eh + el)) = expf(-eh) (1 - el), so the
// factor keeps FP32 relative accuracy even far in the tails, where the
// exponent is large and a plain FP32 argument would lose ~e * 2^-24.
// Dividing by the value at the midpoint nearest the mean (u0) is a constant
// per (k, d) that the normalisation removes; it keeps narrow densities from
// underflowing.
__device__ __forceinline__ float dens_value(int kind, int64_t a, const GaussArg &ga, double xa, double mu,
                                            double sigma, double tlo, double thi, float &u) {
    if (kind == VUP_UNIFORM) {
        u = 0.f;
        double half = __dmul_rn(0.5, sigma);
        double dx = fabs(__dsub_rn(xa, mu));
        return dx <= half ? 1.f : 0.f;
    }
    // t = (a - n) - f exactly as a pair
    const float A = (float)((double)a - ga.nk);
    float th, tl;
    two_sum(A, -ga.fh, th, tl);
    tl -= ga.fl;
    // u = t r
    const float uh = th * ga.rh;
    const float ul = fmaf(th, ga.rh, -uh) + (th * ga.rl + tl * ga.rh);
    u = uh + ul;
    if (kind == VUP_TRUNCNORM && !(tlo <= xa && xa <= thi)) return 0.f;
    // u^2 - u0^2
    const float sh = uh * uh;
    const float sl = fmaf(uh, uh, -sh) + 2.f * uh * ul;
    float dh, dl;
    two_sum(sh, -ga.qh, dh, dl);
    dl += sl - ga.ql;
    const float eh0 = 0.5f * dh, el0 = 0.5f * dl;
    const float eh = eh0 + el0;
    const float el = el0 - (eh - eh0);
    return expf(-eh) * (1.f - el);
}

__global__ void k_density_prep(DensIn in, int64_t K, int64_t K_pad, int ndim, int64_t n0, int64_t n1,
                               int64_t n2, double lo0, double lo1, double lo2, double h0, double h1,
                               double h2, DensConst *__restrict__ dconst, DensStats *__restrict__ dstats,
                               float *__restrict__ ftab, int *__restrict__ dstatus) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (k >= K_pad) return;
    const int64_t nd = d == 0 ? n0 : (d == 1 ? n1 : n2);
    const double lo = d == 0 ? lo0 : (d == 1 ? lo1 : lo2);
    const double h = d == 0 ? h0 : (d == 1 ? h1 : h2);
    int64_t off = 0;
    if (d >= 1) off += n0 * K_pad;
    if (d >= 2) off += n1 * K_pad;
    float *tab = ftab + off;
    if (k >= K) {
        for (int64_t a = 0; a < nd; ++a) tab[a * K_pad + k] = 0.f;
        return;
    }
    const int64_t p = k * ndim + d;
    const int kind = in.kind[p];
    const double mu = in.mu[p], sigma = in.sigma[p];
    const double tlo = in.lo ? in.lo[p] : 0.0, thi = in.hi ? in.hi[p] : 0.0;
    // index coordinate of the mean: (mu - lo) / h - 1/2 = nk + f
    const double c = (mu - lo) / h - 0.5;
    const double nk = floor(c);
    const double fd = c - nk;
    const double rd = h / sigma;
    const float f = (float)fd;
    const float r = (float)rd;
    GaussArg ga;
    ga.nk = nk;
    ga.fh = f;
    ga.fl = (float)(fd - (double)f);
    ga.rh = r;
    ga.rl = (float)(rd - (double)r);
    // squared index-space distance from the mean to its nearest midpoint
    double anear = floor(c + 0.5);
    anear = fmin(fmax(anear, 0.0), (double)(nd - 1));
    const double u0 = ((anear - nk) - fd) * rd;
    double u0sq = kind == VUP_UNIFORM ? 0.0 : u0 * u0;
    if (!(u0sq < 1e30)) u0sq = 0.0;
    ga.qh = (float)u0sq;
    ga.ql = (float)(u0sq - (double)ga.qh);
    KSum S0, S1, S2;
    for (int64_t a = 0; a < nd; ++a) {
        double xa = 0.0;
        if (kind != VUP_GAUSS) xa = __dadd_rn(lo, __dmul_rn((double)a + 0.5, h));
        float u;
        float g = dens_value(kind, a, ga, xa, mu, sigma, tlo, thi, u);
        tab[a * K_pad + k] = g;
        S0.add(g);
        S1.add(g * u);
        S2.add(g * u * u);
    }
    DensConst dc;
    dc.n = (int32_t)fmax(fmin(nk, 2147483647.0), -2147483647.0);
    dc.f = f;
    dc.r = r;
    dc.kind = kind;
    dconst[p] = dc;
    const double Z = S0.value();
    DensStats ds;
    ds.invZ = Z > 0.0 ? 1.0 / Z : 0.0;
    ds.Eu = Z > 0.0 ? S1.value() / Z : 0.0;
    ds.Eu2 = Z > 0.0 ? S2.value() / Z : 0.0;
    ds.inv_sigma = 1.0 / sigma;
    dstats[p] = ds;
    if (!(Z > 0.0)) atomicCAS(dstatus, 0, VUP_DSTAT_EMPTY);
}

// A-operand table of the tensor-core contraction: rows k, reduction index a
// contiguous (K-major), each FP32 factor split into BF16 hi + lo.
__global__ void k_split_transpose(const float *__restrict__ tab, int64_t nd, int64_t K_pad,
                                  int64_t R_pad, __nv_bfloat16 *__restrict__ hi,
                                  __nv_bfloat16 *__restrict__ lo) {
    __shared__ float t[32][33];
    const int64_t a0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int64_t a = a0 + y, k = k0 + threadIdx.x;
        t[y][threadIdx.x] = (a < nd && k < K_pad) ? tab[a * K_pad + k] : 0.f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int64_t k = k0 + y, a = a0 + threadIdx.x;
        if (k < K_pad && a < R_pad) {
            float v = t[threadIdx.x][y];
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            float rem = v - __bfloat162float(h);
            hi[k * R_pad + a] = h;
            lo[k * R_pad + a] = __float2bfloat16_rn(rem);
        }
    }
}

}  // namespace

size_t vup_ftab_floats(const vup_grid g) {
    size_t s = 0;
    for (int d = 0; d < g->ndim; ++d) s += (size_t)g->n[d];
    return s;
}

// need_bf16_orient_mask: bit o set -> build the split BF16 A table for the
// reduction axis of orientation o.
vup_status vup_density_prep(vup_grid g, const vup_densities *d, int need_bf16_orient_mask, cudaStream_t s) {
    const int64_t K = d->K;
    const int64_t K_pad = ceil_div64(K, 128) * 128;
    DensIn in{d->kind, d->mu, d->sigma, d->lo, d->hi};
    double h[3];
    for (int q = 0; q < 3; ++q) h[q] = (g->hi[q] - g->lo[q]) / (double)g->n[q];
    dim3 grd((unsigned)ceil_div64(K_pad, 128), (unsigned)g->ndim);
    VUP_PROF("density_prep", s, 1 + __builtin_popcount(need_bf16_orient_mask));
    k_density_prep<<<grd, 128, 0, s>>>(in, K, K_pad, g->ndim, g->n[0], g->n[1], g->n[2], g->lo[0], g->lo[1],
                                       g->lo[2], h[0], h[1], h[2], (DensConst *)g->dconst.p,
                                       (DensStats *)g->dstats.p, (float *)g->ftab.p, g->dstatus);
    VUP_CHECK_LAUNCH();
    for (int o = 0; o < 2; ++o) {
        if (!(need_bf16_orient_mask & (1 << o))) continue;
        const Orient &ori = g->orient[o];
        const int dred = ori.red_axis0;
        int64_t off = 0;
        for (int q = 0; q < dred; ++q) off += g->n[q] * K_pad;
        __nv_bfloat16 *hi = (__nv_bfloat16 *)g->atab_hi.p + (size_t)o * K_pad * ori.R_pad * 0;
        __nv_bfloat16 *lo = (__nv_bfloat16 *)g->atab_lo.p;
        if (o == 1) {
            // orientation-1 tables live after the orientation-0 tables
            const size_t o0 = (size_t)K_pad * g->orient[0].R_pad;
            hi = (__nv_bfloat16 *)g->atab_hi.p + o0;
            lo = (__nv_bfloat16 *)g->atab_lo.p + o0;
        }
        dim3 tg((unsigned)ceil_div64(ori.R_pad, 32), (unsigned)ceil_div64(K_pad, 32));
        k_split_transpose<<<tg, dim3(32, 8), 0, s>>>((const float *)g->ftab.p + off, g->n[dred], K_pad, ori.R_pad,
                                                     hi, lo);
        VUP_CHECK_LAUNCH();
    }
    return VUP_OK;
}
