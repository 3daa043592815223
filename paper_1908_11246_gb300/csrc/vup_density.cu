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
#include <vector>

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

// Unnormalised Gaussian factor at index offset A = a - n (an integer held
// exactly in FP32), and u = (A - f) r, the midpoint's distance from the mean
// in units of sigma.  The exponent 0.5 (u^2 - u0^2) is carried as an FP32
// pair (error ~2^-44 relative) and exp is split, exp(-(eh + el)) =
// expf(-eh) (1 - el), so the factor keeps FP32 relative accuracy even far in
// the tails, where the exponent is large and a plain FP32 argument would lose
// ~e * 2^-24.  Dividing by the value at the midpoint nearest the mean (u0) is
// a constant per (k, d) that the normalisation removes; it keeps narrow
// densities from underflowing.
__device__ __forceinline__ float gauss_value(float A, const GaussArg &ga, float &u) {
    // t = A - f exactly as a pair
    float th, tl;
    two_sum(A, -ga.fh, th, tl);
    tl -= ga.fl;
    // u = t r
    const float uh = th * ga.rh;
    const float ul = fmaf(th, ga.rh, -uh) + (th * ga.rl + tl * ga.rh);
    u = uh + ul;
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

// Midpoint coordinate of cell a, x_a = lo + (a + 1/2) h, rounded in FP64 in
// this order (the support decisions below compare it with FP64 bounds).
__device__ __forceinline__ double midpoint(double lo, double h, int64_t a) {
    return __dadd_rn(lo, __dmul_rn((double)a + 0.5, h));
}

// First a in [b, e) with pred(a) true, e if none, for a predicate that is
// false then true along a (binary search: a few FP64 evaluations per segment
// instead of one per point).
template <class P>
__device__ __forceinline__ int64_t first_true(int64_t b, int64_t e, P pred) {
    while (b < e) {
        const int64_t m = b + ((e - b) >> 1);
        if (pred(m)) e = m; else b = m + 1;
    }
    return b;
}

// Factor values of one thread's segment [a_begin, a_end) of axis cells,
// written to tab (stride K_pad) and summed (compensated) into S0 = sum g,
// S1 = sum g u, S2 = sum g u^2.  Cells in [in_b, in_e) are inside the
// support (uniform: g = 1 there; truncated normal: the Gaussian there, 0
// outside).  EXACT_F32: every a - n in the segment is below 2^24 in
// magnitude, so A is carried as an FP32 counter; otherwise A is rounded
// from FP64 per cell.
template <bool EXACT_F32, bool STATS>
__device__ __forceinline__ void prep_segment(float *__restrict__ tab, int64_t K_pad, int kind, int64_t a_begin,
                                             int64_t a_end, int64_t in_b, int64_t in_e, const GaussArg &ga,
                                             KSum &S0, KSum &S1, KSum &S2) {
    float Af = (float)((double)a_begin - ga.nk);
    for (int64_t a = a_begin; a < a_end; ++a) {
        const float A = EXACT_F32 ? Af : (float)((double)a - ga.nk);
        Af += 1.f;
        float u;
        const float gv = gauss_value(A, ga, u);
        const bool inside = a >= in_b && a < in_e;
        float g;
        if (kind == VUP_UNIFORM) {
            g = inside ? 1.f : 0.f;
            u = 0.f;
        } else {
            g = (kind == VUP_TRUNCNORM && !inside) ? 0.f : gv;
        }
        tab[a * K_pad] = g;
        S0.add(g);
        if (STATS) {
            S1.add(g * u);
            S2.add(g * u * u);
        }
    }
}

// Everything one density-prep launch needs for one grid (one instance).
struct DensJob {
    DensIn in;
    int64_t K, K_pad;
    int ndim;
    int64_t n[3];
    double lo[3], h[3];
    int S;  // segments per axis
    DensConst *dconst;
    double *dpart;
    float *ftab;
    DensStats *dstats;
    int *dstatus;
    // split BF16 A table of the orientation-0 reduction axis (tensor-core path)
    const float *red_tab;
    int64_t nd_red, R_pad;
    __nv_bfloat16 *ahi, *alo;
};

// Density factors of densities kb*128 .. kb*128+127 on axis d, segment z of
// that axis: the factor table entries and partial compensated sums.
template <bool STATS>
__device__ __forceinline__ void density_prep_body(const DensJob &J, int64_t kb, int d, int z) {
    const int64_t k = kb * (int64_t)blockDim.x + threadIdx.x;
    if (k >= J.K_pad) return;
    const int64_t K = J.K, K_pad = J.K_pad;
    const int ndim = J.ndim, S = J.S;
    const DensIn &in = J.in;
    const int64_t nd = J.n[d];
    // this thread's segment of the axis
    const int64_t seg = (nd + S - 1) / S;
    const int64_t a_begin = z * seg, a_end = a_begin + seg < nd ? a_begin + seg : nd;
    const double lo = J.lo[d];
    const double h = J.h[d];
    int64_t off = 0;
    for (int q = 0; q < d; ++q) off += J.n[q] * K_pad;
    float *tab = J.ftab + off;
    if (k >= K) {
        for (int64_t a = a_begin; a < a_end; ++a) tab[a * K_pad + k] = 0.f;
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
    // support of a uniform or truncated density: an interval of cells, since
    // x_a is non-decreasing in a
    int64_t in_b = a_begin, in_e = a_end;
    if (kind == VUP_UNIFORM) {
        const double half = __dmul_rn(0.5, sigma);
        in_b = first_true(a_begin, a_end, [&](int64_t a) { return __dsub_rn(midpoint(lo, h, a), mu) >= -half; });
        in_e = first_true(in_b, a_end, [&](int64_t a) { return !(__dsub_rn(midpoint(lo, h, a), mu) <= half); });
    } else if (kind == VUP_TRUNCNORM) {
        in_b = first_true(a_begin, a_end, [&](int64_t a) { return midpoint(lo, h, a) >= tlo; });
        in_e = first_true(in_b, a_end, [&](int64_t a) { return !(midpoint(lo, h, a) <= thi); });
    }
    KSum S0, S1, S2;
    const double A0 = (double)a_begin - nk;
    if (fabs(A0) + (double)(a_end - a_begin) < 16777216.0)
        prep_segment<true, STATS>(tab + k, K_pad, kind, a_begin, a_end, in_b, in_e, ga, S0, S1, S2);
    else
        prep_segment<false, STATS>(tab + k, K_pad, kind, a_begin, a_end, in_b, in_e, ga, S0, S1, S2);
    if (z == 0) {
        DensConst dc;
        dc.n = (int32_t)fmax(fmin(nk, 2147483647.0), -2147483647.0);
        dc.f = f;
        dc.r = r;
        dc.kind = kind;
        J.dconst[p] = dc;
    }
    double *q = J.dpart + (((int64_t)d * S + z) * K_pad + k) * 3;
    q[0] = S0.value();
    q[1] = S1.value();
    q[2] = S2.value();
}


// Normalisation statistics from the per-segment compensated sums (segments
// added in order, FP64): Z = sum g, E[u] and E[u^2] under g / Z.
__device__ __forceinline__ void density_finish_body(const DensJob &J, int64_t kb, int d) {
    const int64_t k = kb * (int64_t)blockDim.x + threadIdx.x;
    if (k >= J.K) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int z = 0; z < J.S; ++z) {
        const double *q = J.dpart + (((int64_t)d * J.S + z) * J.K_pad + k) * 3;
        s0 += q[0];
        s1 += q[1];
        s2 += q[2];
    }
    const int64_t p = k * J.ndim + d;
    DensStats ds;
    ds.invZ = s0 > 0.0 ? 1.0 / s0 : 0.0;
    ds.Eu = s0 > 0.0 ? s1 / s0 : 0.0;
    ds.Eu2 = s0 > 0.0 ? s2 / s0 : 0.0;
    ds.inv_sigma = 1.0 / J.in.sigma[p];
    J.dstats[p] = ds;
    if (!(s0 > 0.0)) atomicCAS(J.dstatus, 0, VUP_DSTAT_EMPTY);
}

// A-operand table of the tensor-core contraction: rows k, reduction index a
// contiguous (K-major), each FP32 factor split into BF16 hi + lo (see
// split_transpose_body for the tiling).
// Split of one FP32 value into hi + lo: BF16 pair (tensor kind::f16) or
// TF32 pair stored in floats (kind::tf32).
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Two consecutive reduction indices of one density row split together (one
// 4-byte BF16 pair or 8-byte TF32 pair store per array).
__device__ __forceinline__ void split_store2(__nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t i, float v0, float v1) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
    *reinterpret_cast<__nv_bfloat162 *>(hi + i) = __halves2bfloat162(h0, h1);
    *reinterpret_cast<__nv_bfloat162 *>(lo + i) = __halves2bfloat162(__float2bfloat16_rn(v0 - __bfloat162float(h0)),
                                                                     __float2bfloat16_rn(v1 - __bfloat162float(h1)));
}
__device__ __forceinline__ void split_store2(float *hi, float *lo, int64_t i, float v0, float v1) {
    const float h0 = to_tf32(v0), h1 = to_tf32(v1);
    *reinterpret_cast<float2 *>(hi + i) = make_float2(h0, h1);
    *reinterpret_cast<float2 *>(lo + i) = make_float2(to_tf32(v0 - h0), to_tf32(v1 - h1));
}

// Block (bx, by) transposes the 64 (a) x 128 (k) tile at a = 64 bx,
// k = 128 by: the 64 rows are read with 16-byte loads (eight per thread, in
// flight together), then each lane writes two consecutive a of one density
// row.  R_pad is a multiple of 64, K_pad of 128.
constexpr int kSplitK = 128;
template <typename T>
__device__ __forceinline__ void split_transpose_body(const float *__restrict__ tab, int64_t nd, int64_t K_pad,
                                                     int64_t R_pad, T *__restrict__ hi, T *__restrict__ lo,
                                                     int64_t bx, int64_t by) {
    __shared__ float t[64][kSplitK + 1];
    const int64_t a0 = bx * 64, k0 = by * kSplitK;
    float4 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t a = a0 + threadIdx.y + 8 * i;
        v[i] = a < nd ? *reinterpret_cast<const float4 *>(tab + a * K_pad + k0 + 4 * threadIdx.x)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float *r = &t[threadIdx.y + 8 * i][4 * threadIdx.x];
        r[0] = v[i].x;
        r[1] = v[i].y;
        r[2] = v[i].z;
        r[3] = v[i].w;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < kSplitK; y += blockDim.y) {
        const int64_t k = k0 + y, a = a0 + 2 * threadIdx.x;
        split_store2(hi, lo, k * R_pad + a, t[2 * threadIdx.x][y], t[2 * threadIdx.x + 1][y]);
    }
    __syncthreads();
}

// STATS: also the sums of g u and g u^2 (E[u], E[u^2] of the IPSA derivatives)
template <bool STATS>
__global__ void k_density_prep(DensJob J) {
    pdl_trigger();
    pdl_wait();
    density_prep_body<STATS>(J, blockIdx.x, blockIdx.y, blockIdx.z);
}
__global__ void k_density_finish(DensJob J) {
    pdl_trigger();
    pdl_wait();
    density_finish_body(J, blockIdx.x, blockIdx.y);
}
// grid: x = density tiles of 128 (more than the 65535 limit of y for large K), y = axis tiles
template <typename T>
__global__ void k_split_transpose(const float *__restrict__ tab, int64_t nd, int64_t K_pad, int64_t R_pad,
                                  T *__restrict__ hi, T *__restrict__ lo) {
    pdl_trigger();
    pdl_wait();
    split_transpose_body<T>(tab, nd, K_pad, R_pad, hi, lo, blockIdx.y, blockIdx.x);
}

// Batched forms: one launch for the blocks of every instance; items[b] =
// (instance, block coordinates) of block b.
__global__ void k_density_prep_batched(const DensJob *__restrict__ jobs, const int4 *__restrict__ items) {
    const int4 it = items[blockIdx.x];
    density_prep_body<false>(jobs[it.x], it.y, it.z, it.w);
}
__global__ void k_density_finish_batched(const DensJob *__restrict__ jobs, const int4 *__restrict__ items) {
    const int4 it = items[blockIdx.x];
    density_finish_body(jobs[it.x], it.y, it.z);
}
__global__ void k_split_transpose_batched(const DensJob *__restrict__ jobs, const int4 *__restrict__ items) {
    const int4 it = items[blockIdx.x];
    const DensJob &J = jobs[it.x];
    split_transpose_body<__nv_bfloat16>(J.red_tab, J.nd_red, J.K_pad, J.R_pad, J.ahi, J.alo, it.y, it.z);
}

int density_segments(vup_grid g) {
    int64_t nmax = 1;
    for (int q = 0; q < g->ndim; ++q) nmax = std::max(nmax, g->n[q]);
    return (int)std::max<int64_t>(1, std::min<int64_t>(16, nmax / 128));
}

DensJob make_job(vup_grid g, const vup_densities *d) {
    DensJob J{};
    J.in = DensIn{d->kind, d->mu, d->sigma, d->lo, d->hi};
    J.K = d->K;
    J.K_pad = ceil_div64(d->K, 128) * 128;
    J.ndim = g->ndim;
    for (int q = 0; q < 3; ++q) {
        J.n[q] = g->n[q];
        J.lo[q] = g->lo[q];
        J.h[q] = (g->hi[q] - g->lo[q]) / (double)g->n[q];
    }
    J.S = density_segments(g);
    J.dconst = (DensConst *)g->dconst.p;
    J.dpart = (double *)g->dpart.p;
    J.ftab = (float *)g->ftab.p;
    J.dstats = (DensStats *)g->dstats.p;
    J.dstatus = g->dstatus;
    const Orient &o = g->orient[0];
    int64_t off = 0;
    for (int q = 0; q < o.red_axis0; ++q) off += g->n[q] * J.K_pad;
    J.red_tab = (const float *)g->ftab.p + off;
    J.nd_red = g->n[o.red_axis0];
    J.R_pad = o.R_pad;
    J.ahi = (__nv_bfloat16 *)g->atab_hi.p;
    J.alo = (__nv_bfloat16 *)g->atab_lo.p;
    return J;
}

}  // namespace

size_t vup_ftab_floats(const vup_grid g) {
    size_t s = 0;
    for (int d = 0; d < g->ndim; ++d) s += (size_t)g->n[d];
    return s;
}

vup_status vup_density_reserve(vup_grid g, int64_t K) {
    const int64_t K_pad = ceil_div64(K, 128) * 128;
    return devbuf_reserve(g->dpart, sizeof(double) * 3 * (size_t)density_segments(g) * g->ndim * K_pad);
}

// need_bf16_orient_mask: bit o set -> build the split BF16 A table for the
// reduction axis of orientation o.
template <typename T>
static vup_status split_tables(vup_grid g, int mask, int64_t K_pad, T *hi0, T *lo0, cudaStream_t s);

vup_status vup_density_prep(vup_grid g, const vup_densities *d, int need_bf16_orient_mask, cudaStream_t s,
                            bool tf32, bool stats) {
    vup_status st = vup_density_reserve(g, d->K);
    if (st != VUP_OK) return st;
    const DensJob J = make_job(g, d);
    const int64_t K_pad = J.K_pad;
    dim3 grd((unsigned)ceil_div64(K_pad, 128), (unsigned)g->ndim, (unsigned)J.S);
    VUP_PROF("density_prep", s, 2 + __builtin_popcount(need_bf16_orient_mask));
    VUP_CHECK_CUDA(stats ? launch_pdl(k_density_prep<true>, grd, 128, 0, s, J)
                         : launch_pdl(k_density_prep<false>, grd, 128, 0, s, J));
    dim3 fgrd((unsigned)ceil_div64(d->K, 128), (unsigned)g->ndim);
    VUP_CHECK_CUDA(launch_pdl(k_density_finish, fgrd, 128, 0, s, J));
    if (tf32) return split_tables<float>(g, need_bf16_orient_mask, K_pad, (float *)g->atf_hi.p,
                                         (float *)g->atf_lo.p, s);
    return split_tables<__nv_bfloat16>(g, need_bf16_orient_mask, K_pad, (__nv_bfloat16 *)g->atab_hi.p,
                                       (__nv_bfloat16 *)g->atab_lo.p, s);
}

// Split tables of the A operand for the orientations in `mask` (T: BF16 or
// TF32-in-float), written to hi / lo.
template <typename T>
static vup_status split_tables(vup_grid g, int mask, int64_t K_pad, T *hi0, T *lo0, cudaStream_t s) {
    for (int o = 0; o < 2; ++o) {
        if (!(mask & (1 << o))) continue;
        const Orient &ori = g->orient[o];
        const int dred = ori.red_axis0;
        int64_t off = 0;
        for (int q = 0; q < dred; ++q) off += g->n[q] * K_pad;
        T *hi = hi0, *lo = lo0;
        if (o == 1) {
            // orientation-1 tables live after the orientation-0 tables
            const size_t o0 = (size_t)K_pad * g->orient[0].R_pad;
            hi += o0;
            lo += o0;
        }
        dim3 tg((unsigned)ceil_div64(K_pad, kSplitK), (unsigned)ceil_div64(ori.R_pad, 64));
        VUP_CHECK_CUDA(launch_pdl(k_split_transpose<T>, tg, dim3(32, 8), 0, s, (const float *)g->ftab.p + off,
                                  (int64_t)g->n[dred], K_pad, ori.R_pad, hi, lo));
    }
    return VUP_OK;
}

// Batched density preparation for n instances (one launch per stage).  The
// job and item tables are built on the host and uploaded into `plan`
// (device memory owned by the caller); returns the device pointers' layout
// via the launch.  Scratch of every grid must already be reserved for its K.
struct DensPlan {
    DevBuf jobs, items;
    int n_prep = 0, n_fin = 0, n_split = 0;
};

vup_status vup_density_plan(int n, const vup_grid *gs, const vup_densities *ds, bool bf16, void **plan_out) {
    DensPlan *P = new DensPlan();
    std::vector<DensJob> jobs(n);
    std::vector<int4> prep, fin, split;
    for (int i = 0; i < n; ++i) {
        jobs[i] = make_job(gs[i], &ds[i]);
        const DensJob &J = jobs[i];
        const int64_t nkb_pad = ceil_div64(J.K_pad, 128), nkb = ceil_div64(J.K, 128);
        for (int d = 0; d < J.ndim; ++d)
            for (int z = 0; z < J.S; ++z)
                for (int64_t kb = 0; kb < nkb_pad; ++kb) prep.push_back(make_int4(i, (int)kb, d, z));
        for (int d = 0; d < J.ndim; ++d)
            for (int64_t kb = 0; kb < nkb; ++kb) fin.push_back(make_int4(i, (int)kb, d, 0));
        if (bf16)
            for (int64_t by = 0; by < ceil_div64(J.K_pad, kSplitK); ++by)
                for (int64_t bx = 0; bx < ceil_div64(J.R_pad, 64); ++bx)
                    split.push_back(make_int4(i, (int)bx, (int)by, 0));
    }
    P->n_prep = (int)prep.size();
    P->n_fin = (int)fin.size();
    P->n_split = (int)split.size();
    std::vector<int4> all;
    all.insert(all.end(), prep.begin(), prep.end());
    all.insert(all.end(), fin.begin(), fin.end());
    all.insert(all.end(), split.begin(), split.end());
    vup_status st;
    if ((st = devbuf_reserve(P->jobs, sizeof(DensJob) * n)) != VUP_OK ||
        (st = devbuf_reserve(P->items, sizeof(int4) * all.size())) != VUP_OK) {
        devbuf_free(P->jobs);
        devbuf_free(P->items);
        delete P;
        return st;
    }
    VUP_CHECK_CUDA(cudaMemcpy(P->jobs.p, jobs.data(), sizeof(DensJob) * n, cudaMemcpyHostToDevice));
    VUP_CHECK_CUDA(cudaMemcpy(P->items.p, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice));
    *plan_out = P;
    return VUP_OK;
}

void vup_density_plan_free(void *plan) {
    DensPlan *P = (DensPlan *)plan;
    if (!P) return;
    devbuf_free(P->jobs);
    devbuf_free(P->items);
    delete P;
}

vup_status vup_density_batched(void *plan, cudaStream_t s) {
    const DensPlan *P = (const DensPlan *)plan;
    const DensJob *jobs = (const DensJob *)P->jobs.p;
    const int4 *items = (const int4 *)P->items.p;
    VUP_PROF("density_prep_batched", s, P->n_split ? 3 : 2);
    if (P->n_prep) k_density_prep_batched<<<P->n_prep, 128, 0, s>>>(jobs, items);
    VUP_CHECK_LAUNCH();
    if (P->n_fin) k_density_finish_batched<<<P->n_fin, 128, 0, s>>>(jobs, items + P->n_prep);
    VUP_CHECK_LAUNCH();
    if (P->n_split) k_split_transpose_batched<<<P->n_split, dim3(32, 8), 0, s>>>(jobs, items + P->n_prep + P->n_fin);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}
