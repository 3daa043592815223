// Moment contraction on CUDA cores in FP32 (the plain FP32 GPU path), and the
// FP64 epilogues shared with the tensor-core path.
//
// For a tensor-product grid with product densities the moments factor:
//   M[k, j] = sum_q g_rest(k, q) sum_r g_red(k, r) Z_j[q, r] / (Z_rest Z_red)
// where r runs over the reduction axis (contiguous in y) and q over the rest.
// The inner sum is a GEMM  T[k, (q, j)] = sum_r A[k, r] B[r, (q, j)]  with
// A = g_red (K x R) and B = the power table (R x 4Q); the epilogue contracts
// T with g_rest on the fly.  W itself (K x N) never exists.  Output moments
// of Eq. VUP's output probability matrix (Fig. 4c expectation fields).
#include "vup_internal.cuh"

#include <math.h>

#include <algorithm>
#include <vector>

namespace {

constexpr int BM = 128, BN = 128, BK = 16;

struct EpiArgs {
    const float *g_rest0;   // factor table of the first rest axis  [n][K_pad]
    const float *g_rest1;   // second rest axis (3-D) or nullptr
    int64_t n_rest1;        // size of the second rest axis (1 if none)
    int64_t Q;              // number of rest points
    const DensConst *dconst;  // for IPSA weights of the rest axis
    int ndim;
    int rest_axis;          // axis index of the (single) rest axis for IPSA
};

// One 128 x 128 output tile: column tile ct, row (density) tile rt.
struct SimtJob {
    const float *A;
    const float *Zt;
    int64_t R, K_pad, ldz;
    EpiArgs ep;
    int64_t n_ct;
    float *part;
};

// Reduction terms summed in one plain FP32 chain before the chain is folded
// into the tile's weighted sums.  Rounding bound of one chain: (kChain - 1)
// eps of the sum of its terms' magnitudes; the fold is compensated (Kahan),
// so the long sums over the reduction axis add only ~2 eps more: the
// contraction stays within ~12 eps (7e-7) of sum_i W |z|^j whatever R is,
// where one chain over the whole axis would grow like sqrt(R) eps.
constexpr int kChain = 8;

// Epilogue weight of rest point q for density k: the rest-axis factor e
// (wmode 0), or e u and e u^2 with u the rest-axis index coordinate's
// distance from the mean in units of sigma (wmode 1, 2: the IPSA sums).
__device__ __forceinline__ float epi_weight(const EpiArgs &ep, int64_t K_pad, int64_t k, int64_t q, int wmode) {
    if (q >= ep.Q) return 0.f;
    int64_t qa = q, qb = 0;
    if (ep.g_rest1) {
        qa = q / ep.n_rest1;
        qb = q - qa * ep.n_rest1;
    }
    float e = ep.g_rest0[qa * K_pad + k];
    if (ep.g_rest1) e *= ep.g_rest1[qb * K_pad + k];
    if (wmode) {
        const DensConst dc = ep.dconst[k * ep.ndim + ep.rest_axis];
        const float u = ((float)(q - dc.n) - dc.f) * dc.r;
        e *= wmode == 1 ? u : u * u;
    }
    return e;
}

// One 128 (densities) x 128 (columns (q, j)) tile.  Each thread owns 8 rows
// x 8 columns (2 rest points x 4 powers): the GEMM part accumulates kChain
// reduction terms per plain FP32 chain, then folds the chain into
// out[row][j] += w(row, q) * chain with Kahan compensation; the 16 column
// threads of a row are reduced in FP64 and the tile writes one FP32 partial
// per (row, power) for the FP64 finish.
__device__ __forceinline__ void simt_tile(const float *__restrict__ A, const float *__restrict__ Zt, int64_t R,
                                          int64_t K_pad, int64_t ldz, const EpiArgs &ep, int64_t n_ct,
                                          float *__restrict__ part, int64_t ct, int64_t row_tile, int wmode) {
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t k0 = row_tile * BM;
    const int64_t c0 = ct * BN;
    auto row_of = [&](int i) { return k0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4)); };

    // epilogue weights of the thread's rows and rest points, fixed for the tile
    float w[8][2];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int gq = 0; gq < 2; ++gq) w[i][gq] = epi_weight(ep, K_pad, row_of(i), c0 / 4 + gq * 16 + tx, wmode);

    float acc[8][8];
    float out[8][4], cmp[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) out[i][j] = cmp[i][j] = 0.f;
    auto fold = [&]() {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int gq = 0; gq < 2; ++gq) {
                    const float yv = fmaf(w[i][gq], acc[i][gq * 4 + j], -cmp[i][j]);
                    const float t = out[i][j] + yv;
                    cmp[i][j] = (t - out[i][j]) - yv;
                    out[i][j] = t;
                }
    };

    float4 ra[2], rb[2];
    auto load_regs = [&](int64_t r0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = tid + h * 256;
            const int row = e >> 5, c4 = e & 31;
            const int64_t r = r0 + row;
            if (r < R) {
                ra[h] = *reinterpret_cast<const float4 *>(A + r * K_pad + k0 + c4 * 4);
                rb[h] = *reinterpret_cast<const float4 *>(Zt + r * ldz + c0 + c4 * 4);
            } else {
                ra[h] = make_float4(0.f, 0.f, 0.f, 0.f);
                rb[h] = ra[h];
            }
        }
    };
    auto store_smem = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = tid + h * 256;
            const int row = e >> 5, c4 = e & 31;
            *reinterpret_cast<float4 *>(&As[buf][row][c4 * 4]) = ra[h];
            *reinterpret_cast<float4 *>(&Bs[buf][row][c4 * 4]) = rb[h];
        }
    };

    const int64_t n_rt = (R + BK - 1) / BK;
    load_regs(0);
    store_smem(0);
    __syncthreads();
    for (int64_t rt = 0; rt < n_rt; ++rt) {
        const int buf = rt & 1;
        if (rt + 1 < n_rt) load_regs((rt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[8], b[8];
            *reinterpret_cast<float4 *>(&a[0]) = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
            *reinterpret_cast<float4 *>(&a[4]) = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
            *reinterpret_cast<float4 *>(&b[0]) = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
            *reinterpret_cast<float4 *>(&b[4]) = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
            if (kk % kChain == 0) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = a[i] * b[j];
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            if (kk % kChain == kChain - 1) fold();
        }
        if (rt + 1 < n_rt) {
            store_smem(buf ^ 1);
        }
        __syncthreads();
    }

    // reduce over the 16 column threads of a half-warp (FP64)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        double v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = (double)out[i][j] - (double)cmp[i][j];
            v[j] += __shfl_xor_sync(0xffffffffu, v[j], 8);
            v[j] += __shfl_xor_sync(0xffffffffu, v[j], 4);
            v[j] += __shfl_xor_sync(0xffffffffu, v[j], 2);
            v[j] += __shfl_xor_sync(0xffffffffu, v[j], 1);
        }
        if (tx == 0)
            *reinterpret_cast<float4 *>(part + (((int64_t)wmode * n_ct + ct) * K_pad + row_of(i)) * 4) =
                make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    }
}

// wmode 0: moments; 1, 2: the IPSA sums with weights e u and e u^2 (one
// launch each, into partial slice wmode).
__global__ void __launch_bounds__(256, 1)
k_moments_simt(const float *__restrict__ A, const float *__restrict__ Zt, int64_t R, int64_t K_pad,
               int64_t ldz, EpiArgs ep, int64_t n_ct, float *__restrict__ part, int wmode) {
    simt_tile(A, Zt, R, K_pad, ldz, ep, n_ct, part, blockIdx.x, blockIdx.y, wmode);
}

// Batched form: one persistent launch over the tiles of many instances,
// longest reductions first (items[t] = (instance, column tile, row tile)).
__global__ void __launch_bounds__(256, 1)
k_moments_simt_batched(const SimtJob *__restrict__ jobs, const int4 *__restrict__ items, int n_items) {
    for (int t = blockIdx.x; t < n_items; t += gridDim.x) {
        const int4 it = items[t];
        const SimtJob J = jobs[it.x];
        simt_tile(J.A, J.Zt, J.R, J.K_pad, J.ldz, J.ep, J.n_ct, J.part, it.y, it.z, 0);
        __syncthreads();
    }
}

// Sum the per-column-tile partials in FP64, undo the normalisation, re-expand
// the moments of z = (y - c) / s into raw moments of y, and form the central
// moments about the mean from the moments of z.
struct FinishJob {
    const float *part;
    int64_t n_ct, K, K_pad;
    int J;
    const DensStats *ds;
    int ndim;
    const double *scale;
    double *raw, *central;
};

__device__ __forceinline__ void moments_finish_body(const float *__restrict__ part, int64_t n_ct, int64_t K,
                                                    int64_t K_pad, int J, const DensStats *__restrict__ ds,
                                                    int ndim, const double *__restrict__ scale,
                                                    double *__restrict__ raw, double *__restrict__ central,
                                                    int64_t kb) {
    const int64_t k = kb * (int64_t)blockDim.x + threadIdx.x;
    if (k >= K) return;
    // the column tiles' partials summed as FP32 TwoSum pairs (about 2^-44
    // relative to the sum of magnitudes, far below the partials' own FP32
    // rounding) on the FP32 pipes, one FP64 conversion per sum: FP64
    // arithmetic runs at a small fraction of the FP32 rate here
    float mh[4] = {0.f, 0.f, 0.f, 0.f}, ml[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int64_t t = 0; t < n_ct; ++t) {
        const float4 v = *reinterpret_cast<const float4 *>(part + (t * K_pad + k) * 4);
        two_sum_acc(mh[0], ml[0], v.x);
        two_sum_acc(mh[1], ml[1], v.y);
        two_sum_acc(mh[2], ml[2], v.z);
        two_sum_acc(mh[3], ml[3], v.w);
    }
    double mz[4];
    for (int j = 0; j < 4; ++j) mz[j] = (double)mh[j] + (double)ml[j];
    double invZ = 1.0;
    for (int d = 0; d < ndim; ++d) invZ *= ds[k * ndim + d].invZ;
    invZ /= scale[kScaleP];  // the tables' power-of-two factor
    for (int j = 0; j < 4; ++j) mz[j] *= invZ;
    const double s = scale[kScaleS], c = scale[kScaleC];
    if (raw) {
        double M[4];
        raw_from_shifted(mz, c, s, M);
        for (int j = 0; j < J; ++j) raw[k * J + j] = M[j];
    }
    if (central) {
        double cm[4];
        central_from_shifted(mz, c, s, cm);
        for (int j = 0; j < J; ++j) central[k * J + j] = cm[j];
    }
}

__global__ void k_moments_finish(const float *__restrict__ part, int64_t n_ct, int64_t K, int64_t K_pad, int J,
                                 const DensStats *__restrict__ ds, int ndim, const double *__restrict__ scale,
                                 double *__restrict__ raw, double *__restrict__ central) {
    pdl_trigger();
    pdl_wait();
    moments_finish_body(part, n_ct, K, K_pad, J, ds, ndim, scale, raw, central, blockIdx.x);
}

__global__ void k_moments_finish_batched(const FinishJob *__restrict__ jobs, const int2 *__restrict__ items) {
    const int2 it = items[blockIdx.x];
    const FinishJob F = jobs[it.x];
    moments_finish_body(F.part, F.n_ct, F.K, F.K_pad, F.J, F.ds, F.ndim, F.scale, F.raw, F.central, it.y);
}

// IPSA combine.  With u_d = (x_d - mu_d) / sigma_d, W = g / sum g and
// z = (y - c) / s, the moments of z have the derivatives
//   dMz_m/dmu_d    = (sum_i W u_d z^m   - E_d[u]   Mz_m) / sigma_d
//   dMz_m/dsigma_d = (sum_i W u_d^2 z^m - E_d[u^2] Mz_m) / sigma_d
// and dM_j/dp = sum_{m=1..j} C(j, m) c^(j-m) s^m dMz_m/dp (Mz_0 = 1 is constant).
// part0 holds orientation 0 (rest = axis 0): [w, w u_0, w u_0^2] partials,
// part1 orientation 1 (rest = axis 1, 2-D only).  A CTA serves 128
// densities with 128 threads per plane q = 3 o + w (orientation o, weight w):
// each sums its plane's column tiles for its density as FP32 TwoSum pairs
// (see moments_finish_body), and the threads of plane 0 combine the six
// sums of their density in FP64.
constexpr int kIpsaFinK = 128;
__global__ void __launch_bounds__(6 * kIpsaFinK) k_ipsa_finish(const float *__restrict__ part0, int64_t nct0,
                                                               const float *__restrict__ part1, int64_t nct1,
                                                               int64_t K, int64_t K_pad, int J,
                                                               const DensStats *__restrict__ ds,
                                                               const DensConst *__restrict__ dc, int ndim,
                                                               const double *__restrict__ scale,
                                                               const double *__restrict__ grad,
                                                               float *__restrict__ dmu, float *__restrict__ dsg) {
    __shared__ double sS[6][kIpsaFinK][4];
    const int kk = threadIdx.x % kIpsaFinK, q = threadIdx.x / kIpsaFinK;
    const int64_t k = blockIdx.x * (int64_t)kIpsaFinK + kk;
    {
        const int o = q / 3, w = q % 3;
        float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
        if (k < K && o < ndim) {
            const float *part = o == 0 ? part0 : part1;
            const int64_t nct = o == 0 ? nct0 : nct1;
#pragma unroll 4
            for (int64_t t = 0; t < nct; ++t) {
                const float4 v = *reinterpret_cast<const float4 *>(part + ((w * nct + t) * K_pad + k) * 4);
                two_sum_acc(sh[0], sl[0], v.x);
                two_sum_acc(sh[1], sl[1], v.y);
                two_sum_acc(sh[2], sl[2], v.z);
                two_sum_acc(sh[3], sl[3], v.w);
            }
        }
        for (int j = 0; j < 4; ++j) sS[q][kk][j] = (double)sh[j] + (double)sl[j];
    }
    __syncthreads();
    if (q != 0 || k >= K) return;
    double invZ = 1.0 / scale[kScaleP];  // the tables' power-of-two factor
    for (int d = 0; d < ndim; ++d) invZ *= ds[k * ndim + d].invZ;
    const double s = scale[kScaleS], c = scale[kScaleC];
    double S[2][3][4];
    for (int o = 0; o < 2; ++o)
        for (int w = 0; w < 3; ++w)
            for (int j = 0; j < 4; ++j) S[o][w][j] = sS[3 * o + w][kk][j];
    for (int d = 0; d < ndim; ++d) {
        const DensStats st = ds[k * ndim + d];
        const bool diff = dc[k * ndim + d].kind != VUP_UNIFORM;
        double dmz[4], dsz[4];
        for (int m = 0; m < 4; ++m) {
            const double Mz = S[0][0][m] * invZ;
            const double Su = S[d][1][m] * invZ;
            const double Su2 = S[d][2][m] * invZ;
            dmz[m] = st.inv_sigma * (Su - st.Eu * Mz);
            dsz[m] = st.inv_sigma * (Su2 - st.Eu2 * Mz);
        }
        // re-expansion without the constant term (c^j of Mz_0 = 1)
        double dM[4], dS[4];
        {
            const double C[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
            for (int j = 1; j <= 4; ++j) {
                double vm = 0.0, vs = 0.0, cp = 1.0;
                for (int m = j; m >= 1; --m) {  // c^(j-m) grows as m falls
                    double sm = 1.0;
                    for (int q = 0; q < m; ++q) sm *= s;
                    vm += C[j][m] * cp * sm * dmz[m - 1];
                    vs += C[j][m] * cp * sm * dsz[m - 1];
                    cp *= c;
                }
                dM[j - 1] = vm;
                dS[j - 1] = vs;
            }
        }
        double gm = 0.0, gs = 0.0;
        for (int j = 0; j < J; ++j) {
            const double dm = diff ? dM[j] : 0.0;
            const double dsd = diff ? dS[j] : 0.0;
            if (grad) {
                gm += grad[k * J + j] * dm;
                gs += grad[k * J + j] * dsd;
            } else {
                dmu[(k * ndim + d) * J + j] = (float)dm;
                dsg[(k * ndim + d) * J + j] = (float)dsd;
            }
        }
        if (grad) {
            dmu[k * ndim + d] = (float)gm;
            dsg[k * ndim + d] = (float)gs;
        }
    }
}

}  // namespace

int64_t vup_simt_col_tiles(const Orient &o) { return ceil_div64(o.NC, BN); }

static EpiArgs epi_for(vup_grid g, int orient, int64_t K_pad) {
    const Orient &o = g->orient[orient];
    EpiArgs ep{};
    auto tab = [&](int axis) {
        int64_t off = 0;
        for (int q = 0; q < axis; ++q) off += g->n[q] * K_pad;
        return (const float *)g->ftab.p + off;
    };
    ep.g_rest0 = tab(o.rest_axes[0]);
    ep.g_rest1 = o.n_rest_axes > 1 ? tab(o.rest_axes[1]) : nullptr;
    ep.n_rest1 = o.n_rest_axes > 1 ? g->n[o.rest_axes[1]] : 1;
    ep.Q = o.Q;
    ep.dconst = (const DensConst *)g->dconst.p;
    ep.ndim = g->ndim;
    ep.rest_axis = o.rest_axes[0];
    return ep;
}

vup_status vup_moments_simt(vup_grid g, int64_t K, int orient, int n_out, float *part, cudaStream_t s) {
    const Orient &o = g->orient[orient];
    const int64_t K_pad = ceil_div64(K, 128) * 128;
    int64_t off = 0;
    for (int q = 0; q < o.red_axis0; ++q) off += g->n[q] * K_pad;
    const float *A = (const float *)g->ftab.p + off;
    const int64_t n_ct = vup_simt_col_tiles(o);
    const int64_t ldz = ceil_div64(o.NC, 128) * 128;
    EpiArgs ep = epi_for(g, orient, K_pad);
    dim3 grd((unsigned)n_ct, (unsigned)(K_pad / BM));
    VUP_PROF(n_out == 1 ? "moments_fp32_simt" : "ipsa_fp32_simt", s, n_out);
    for (int wm = 0; wm < n_out; ++wm) {
        k_moments_simt<<<grd, 256, 0, s>>>(A, g->zs[orient], o.R, K_pad, ldz, ep, n_ct, part, wm);
        VUP_CHECK_LAUNCH();
    }
    return VUP_OK;
}

vup_status vup_moments_finish(vup_grid g, int64_t K, int n_col_tiles, double *raw, double *central,
                              cudaStream_t s, const float *part) {
    const int64_t K_pad = ceil_div64(K, 128) * 128;
    VUP_PROF("moments_finish_fp64", s, 1);
    VUP_CHECK_CUDA(launch_pdl(k_moments_finish, dim3((unsigned)ceil_div64(K, 128)), dim3(128), 0, s,
                              part ? part : (const float *)g->partials.p, (int64_t)n_col_tiles, K, K_pad, g->J,
                              (const DensStats *)g->dstats.p, g->ndim, (const double *)g->ydev_scale, raw, central));
    return VUP_OK;
}

vup_status vup_ipsa_finish(vup_grid g, int64_t K, int n_tiles0, int n_tiles1, const double *grad, float *dmu,
                           float *dsg, cudaStream_t s) {
    const int64_t K_pad = ceil_div64(K, 128) * 128;
    const float *p0 = (const float *)g->ipsa_part.p;
    const float *p1 = p0 + (size_t)3 * n_tiles0 * K_pad * 4;
    VUP_PROF("ipsa_finish_fp64", s, 1);
    k_ipsa_finish<<<(unsigned)ceil_div64(K, kIpsaFinK), 6 * kIpsaFinK, 0, s>>>(
        p0, n_tiles0, p1, n_tiles1, K, K_pad, g->J, (const DensStats *)g->dstats.p,
        (const DensConst *)g->dconst.p, g->ndim, g->ydev_scale, grad, dmu, dsg);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}

// Batched FP32 contraction over n 2-D instances (orientation 0): instance i
// writes its partials [n_ct][K_pad][4] to parts[i]; tiles of the longest
// reductions first.
struct SimtPlan {
    DevBuf jobs, items;
    int n_items = 0;
};

vup_status vup_simt_plan(int n, const vup_grid *gs, const int64_t *Ks, float *const *parts, void **out) {
    std::vector<SimtJob> jobs(n);
    std::vector<std::pair<int64_t, int4>> work;
    for (int i = 0; i < n; ++i) {
        vup_grid g = gs[i];
        const Orient &o = g->orient[0];
        const int64_t K_pad = ceil_div64(Ks[i], 128) * 128;
        int64_t off = 0;
        for (int q = 0; q < o.red_axis0; ++q) off += g->n[q] * K_pad;
        SimtJob &J = jobs[i];
        J.A = (const float *)g->ftab.p + off;
        J.Zt = g->zs[0];
        J.R = o.R;
        J.K_pad = K_pad;
        J.ldz = ceil_div64(o.NC, 128) * 128;
        J.ep = epi_for(g, 0, K_pad);
        J.n_ct = vup_simt_col_tiles(o);
        J.part = parts[i];
        for (int64_t rt = 0; rt < K_pad / BM; ++rt)
            for (int64_t ct = 0; ct < J.n_ct; ++ct) work.push_back({o.R, make_int4(i, (int)ct, (int)rt, 0)});
    }
    std::stable_sort(work.begin(), work.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::vector<int4> items(work.size());
    for (size_t q = 0; q < work.size(); ++q) items[q] = work[q].second;
    SimtPlan *P = new SimtPlan();
    P->n_items = (int)items.size();
    vup_status st;
    if ((st = devbuf_reserve(P->jobs, sizeof(SimtJob) * n)) != VUP_OK ||
        (st = devbuf_reserve(P->items, sizeof(int4) * std::max<size_t>(1, items.size()))) != VUP_OK) {
        devbuf_free(P->jobs);
        devbuf_free(P->items);
        delete P;
        return st;
    }
    VUP_CHECK_CUDA(cudaMemcpy(P->jobs.p, jobs.data(), sizeof(SimtJob) * n, cudaMemcpyHostToDevice));
    VUP_CHECK_CUDA(cudaMemcpy(P->items.p, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    *out = P;
    return VUP_OK;
}

void vup_simt_plan_free(void *plan) {
    SimtPlan *P = (SimtPlan *)plan;
    if (!P) return;
    devbuf_free(P->jobs);
    devbuf_free(P->items);
    delete P;
}

vup_status vup_simt_batched(void *plan, cudaStream_t s) {
    const SimtPlan *P = (const SimtPlan *)plan;
    if (P->n_items == 0) return VUP_OK;
    const int grid = std::min(P->n_items, 2 * vup_num_sms());
    VUP_PROF("moments_fp32_simt_batched", s, 1);
    k_moments_simt_batched<<<grid, 256, 0, s>>>((const SimtJob *)P->jobs.p, (const int4 *)P->items.p, P->n_items);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}

// Batched FP64 finish: instance i sums n_cts[i] column-tile partials from
// parts[i] into raws[i] / centrals[i] (either may be null).
struct FinishPlan {
    DevBuf jobs, items;
    int n_items = 0;
};

vup_status vup_finish_plan(int n, const vup_grid *gs, const int64_t *Ks, const int64_t *n_cts,
                           float *const *parts, double *const *raws, double *const *centrals, void **out) {
    std::vector<FinishJob> jobs(n);
    std::vector<int2> items;
    for (int i = 0; i < n; ++i) {
        vup_grid g = gs[i];
        FinishJob &F = jobs[i];
        F.part = parts[i];
        F.n_ct = n_cts[i];
        F.K = Ks[i];
        F.K_pad = ceil_div64(Ks[i], 128) * 128;
        F.J = g->J;
        F.ds = (const DensStats *)g->dstats.p;
        F.ndim = g->ndim;
        F.scale = g->ydev_scale;
        F.raw = raws ? raws[i] : nullptr;
        F.central = centrals ? centrals[i] : nullptr;
        if (!F.raw && !F.central) continue;
        for (int64_t kb = 0; kb < ceil_div64(Ks[i], 128); ++kb) items.push_back(make_int2(i, (int)kb));
    }
    FinishPlan *P = new FinishPlan();
    P->n_items = (int)items.size();
    vup_status st;
    if ((st = devbuf_reserve(P->jobs, sizeof(FinishJob) * n)) != VUP_OK ||
        (st = devbuf_reserve(P->items, sizeof(int2) * std::max<size_t>(1, items.size()))) != VUP_OK) {
        devbuf_free(P->jobs);
        devbuf_free(P->items);
        delete P;
        return st;
    }
    VUP_CHECK_CUDA(cudaMemcpy(P->jobs.p, jobs.data(), sizeof(FinishJob) * n, cudaMemcpyHostToDevice));
    if (!items.empty())
        VUP_CHECK_CUDA(cudaMemcpy(P->items.p, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
    *out = P;
    return VUP_OK;
}

void vup_finish_plan_free(void *plan) {
    FinishPlan *P = (FinishPlan *)plan;
    if (!P) return;
    devbuf_free(P->jobs);
    devbuf_free(P->items);
    delete P;
}

vup_status vup_finish_batched(void *plan, cudaStream_t s) {
    const FinishPlan *P = (const FinishPlan *)plan;
    if (P->n_items == 0) return VUP_OK;
    VUP_PROF("moments_finish_fp64_batched", s, 1);
    k_moments_finish_batched<<<P->n_items, 128, 0, s>>>((const FinishJob *)P->jobs.p, (const int2 *)P->items.p);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}
