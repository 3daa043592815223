// Coarse-grained IPSA quantities (Sec. 5.2): the estimated values y(l) at
// the densities' centres, the deviation moments about them (Eq. IPSAvar:
// the local expected square deviation Delta^2 is half the second one), the
// IPSA probability matrix (Eq. IPSA: every column of the output probability
// matrix translated by -y(l) onto one grid of deviations) and per-column
// fields (maximum-probability bin, confidence interval) with the global
// vector marginalised over l.  All of it is O(K (B + J)) work on outputs of
// vup_propagate; every decision that yields an integer (a deviation bin, an
// argmax, an interval bound) is taken in FP64 with correctly rounded
// operations in the order the definitions state them.
#include "vup_internal.cuh"

#include <math.h>

#include <algorithm>

namespace {

__device__ __forceinline__ double ext_value(unsigned long long k) {  // ordered key -> double
    const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)u);
}

// Deviation bin of output bin b: floor((c_b - yref - dlo) / wd), clamped.
__device__ __forceinline__ int dev_bin(int b, double ymin, double w, double yref, double dlo, double wd, int nd) {
    const double t = __dadd_rn((double)b, 0.5);
    const double c = __dadd_rn(ymin, __dmul_rn(t, w));
    const double dy = __dsub_rn(c, yref);
    const double f = floor(__ddiv_rn(__dsub_rn(dy, dlo), wd));
    return f < 0.0 ? 0 : (f > (double)(nd - 1) ? nd - 1 : (int)f);
}

// One CTA per column k: every output bin's deviation bin is computed once
// into shared memory (one FP64 division each); the map is non-decreasing in
// b, so the bins of deviation bin e form one contiguous range, found by
// binary search over the shared map and summed in increasing b.
__global__ void k_ipsa_matrix(const float *__restrict__ H, int64_t K, int B, const unsigned long long *__restrict__ ext,
                              const double *__restrict__ yref, int nd, double dlo, double dhi,
                              float *__restrict__ out) {
    extern __shared__ int emap[];  // [B]
    const double ymin = ext_value(ext[0]), ymax = ext_value(ext[1]);
    const double w = __ddiv_rn(__dsub_rn(ymax, ymin), (double)B);
    const double wd = __ddiv_rn(__dsub_rn(dhi, dlo), (double)nd);
    for (int64_t k = blockIdx.x; k < K; k += gridDim.x) {
        const double yr = yref[k];
        __syncthreads();  // the previous column's readers are done
        for (int b = threadIdx.x; b < B; b += blockDim.x) emap[b] = dev_bin(b, ymin, w, yr, dlo, wd, nd);
        __syncthreads();
        const float *h = H + k * B;
        for (int e = threadIdx.x; e < nd; e += blockDim.x) {
            int lo = 0, hi = B;  // first b with emap[b] >= e
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (emap[mid] >= e) hi = mid; else lo = mid + 1;
            }
            double s = 0.0;
            for (int b = lo; b < B && emap[b] == e; ++b) s = __dadd_rn(s, (double)h[b]);
            out[k * nd + e] = (float)s;
        }
    }
}

// out[k][j-1] = sum_{m=0..j} C(j,m) M_m (-yref)^(j-m), M_0 = 1 (FP64).
__global__ void k_deviation_moments(const double *__restrict__ raw, int64_t K, int J,
                                    const double *__restrict__ yref, double *__restrict__ out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= K) return;
    double M[5] = {1.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = 1; j <= J; ++j) M[j] = raw[k * J + j - 1];
    const double c = -yref[k];
    for (int j = 1; j <= J; ++j) {
        double s = 0.0, binom = 1.0, cp = 1.0;
        // terms m = j, j-1, ..., 0: C(j, m) M_m c^(j-m)
        for (int m = j; m >= 0; --m) {
            s += binom * M[m] * cp;
            cp *= c;
            binom = binom * (double)m / (double)(j - m + 1);
        }
        out[k * J + j - 1] = s;
    }
}

// One lane per row k (a warp serves 32 rows): 32 x 32 tiles of the rows are
// staged through shared memory so that the loads stay coalesced, and every
// lane walks its own row in bin order, so the FP32 sums and the decisions
// follow the definitions' sequential order exactly.
__global__ void __launch_bounds__(128) k_sa_rows(const float *__restrict__ H, int64_t K, int nb, double level,
                                                 int32_t *__restrict__ argmax, int32_t *__restrict__ ci) {
    __shared__ float tile[4][32][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k0 = ((int64_t)blockIdx.x * 4 + warp) * 32;
    if (k0 >= K) return;
    float(*t)[33] = tile[warp];
    const int64_t k = k0 + lane;
    auto stage = [&](int b0) {  // t[r][i] = H[k0 + r][b0 + i], all 32 loads in flight
        float v[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = (k0 + r < K && b0 + lane < nb) ? __ldg(H + (k0 + r) * nb + b0 + lane) : 0.f;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 32; ++r) t[r][lane] = v[r];
        __syncwarp();
    };
    const float lo_q = (float)__dmul_rn(0.5, __dsub_rn(1.0, level)), hi_q = (float)__dmul_rn(0.5, __dadd_rn(1.0, level));
    int am = 0;
    float best = 0.f, total = 0.f;
    for (int b0 = 0; b0 < nb; b0 += 32) {
        stage(b0);
        const int m = min(32, nb - b0);
        if (b0 == 0) best = t[lane][0];
        for (int i = 0; i < m; ++i) {
            const float v = t[lane][i];
            if (v > best) {
                best = v;
                am = b0 + i;
            }
            total = __fadd_rn(total, v);
        }
    }
    const float tl = __fmul_rn(lo_q, total), th = __fmul_rn(hi_q, total);
    float cum = 0.f;
    int lo = nb - 1, hi = nb - 1;
    bool have_lo = false, have_hi = false;
    for (int b0 = 0; b0 < nb; b0 += 32) {
        stage(b0);
        const int m = min(32, nb - b0);
        for (int i = 0; i < m; ++i) {
            cum = __fadd_rn(cum, t[lane][i]);
            if (!have_lo && cum > tl) { lo = b0 + i; have_lo = true; }
            if (!have_hi && cum >= th) { hi = b0 + i; have_hi = true; }
        }
    }
    if (k < K) {
        if (argmax) argmax[k] = am;
        if (ci) {
            ci[2 * k] = lo;
            ci[2 * k + 1] = hi;
        }
    }
}

// global[b] = sum_k rho_k H[k][b] / sum_k rho_k (uniform rho when null), in
// two deterministic passes: blocks of kSaRows rows summed in row order into
// partials, then the partials in block order.
constexpr int kSaRows = 64;
__global__ void k_sa_global_part(const float *__restrict__ H, int64_t K, int nb, const double *__restrict__ rho,
                                 double *__restrict__ part, double *__restrict__ rpart) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.y * kSaRows, k1 = min(K, k0 + kSaRows);
    if (b < nb) {
        double g = 0.0;
#pragma unroll 16
        for (int64_t k = k0; k < k1; ++k) g = __dadd_rn(g, __dmul_rn(rho ? rho[k] : 1.0, (double)__ldg(H + k * nb + b)));
        part[(int64_t)blockIdx.y * nb + b] = g;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double rs = 0.0;
        for (int64_t k = k0; k < k1; ++k) rs = __dadd_rn(rs, rho ? rho[k] : 1.0);
        rpart[blockIdx.y] = rs;
    }
}
__global__ void k_sa_global_sum(const double *__restrict__ part, const double *__restrict__ rpart, int64_t nblk,
                                int nb, double *__restrict__ global) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double g = 0.0, rs = 0.0;
    for (int64_t q = 0; q < nblk; ++q) {
        g = __dadd_rn(g, part[q * nb + b]);
        rs = __dadd_rn(rs, rpart[q]);
    }
    global[b] = rs > 0.0 ? __ddiv_rn(g, rs) : g;
}

DevBuf g_sa_part;  // process-wide scratch of the marginalisation

}  // namespace

extern "C" vup_status vup_model_at(vup_grid g, int64_t K, const double *x, double *y, vup_stream_t stream) {
    if (!g || !x || !y || K < 1) return VUP_ERR_INVALID_ARG;
    if (!g->have_model || g->model_id == 0) return VUP_ERR_STATE;
    return vup_launch_model_at(g, K, x, y, (cudaStream_t)stream);
}

extern "C" vup_status vup_deviation_moments(vup_grid g, int64_t K, const double *moments_raw, const double *y_ref,
                                            double *out, vup_stream_t stream) {
    if (!g || !moments_raw || !y_ref || !out || K < 1) return VUP_ERR_INVALID_ARG;
    if (!g->have_model) return VUP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    VUP_PROF("deviation_moments", s, 1);
    k_deviation_moments<<<(unsigned)ceil_div64(K, 128), 128, 0, s>>>(moments_raw, K, g->J, y_ref, out);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}

extern "C" vup_status vup_ipsa_matrix(vup_grid g, int64_t K, const float *hist, const double *y_ref, int n_dbins,
                                      double dlo, double dhi, float *out, vup_stream_t stream) {
    if (!g || !hist || !y_ref || !out || K < 1 || K > VUP_MAX_DENSITIES || n_dbins < 1 || n_dbins > VUP_MAX_BINS)
        return VUP_ERR_INVALID_ARG;
    if (!isfinite(dlo) || !isfinite(dhi) || !(dlo < dhi)) return VUP_ERR_INVALID_ARG;
    if (!g->have_model) return VUP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    VUP_PROF("ipsa_matrix", s, 1);
    const size_t smem = sizeof(int) * (size_t)g->B;
    if (smem > 48 * 1024)
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_ipsa_matrix, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = (unsigned)std::min<int64_t>(K, (int64_t)vup_num_sms() * 8);
    k_ipsa_matrix<<<grid, 256, smem, s>>>(hist, K, g->B, g->ext, y_ref, n_dbins, dlo, dhi, out);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}

extern "C" vup_status vup_sa_fields(int64_t K, int n_bins, const float *hist, double level, const double *rho,
                                    int32_t *argmax, int32_t *ci, double *global, vup_stream_t stream) {
    if (!hist || K < 1 || n_bins < 1 || !(level > 0.0 && level < 1.0)) return VUP_ERR_INVALID_ARG;
    if (!argmax && !ci && !global) return VUP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    VUP_PROF("sa_fields", s, (argmax || ci ? 1 : 0) + (global ? 2 : 0));
    if (argmax || ci) {
        k_sa_rows<<<(unsigned)ceil_div64(K, 128), 128, 0, s>>>(hist, K, n_bins, level, argmax, ci);
        VUP_CHECK_LAUNCH();
    }
    if (global) {
        const int64_t nblk = ceil_div64(K, kSaRows);
        if (nblk > 65535) return VUP_ERR_UNSUPPORTED;
        const vup_status st = devbuf_reserve(g_sa_part, sizeof(double) * (size_t)nblk * (n_bins + 1));
        if (st != VUP_OK) return st;
        double *part = (double *)g_sa_part.p, *rpart = part + (size_t)nblk * n_bins;
        k_sa_global_part<<<dim3((unsigned)ceil_div64(n_bins, 128), (unsigned)nblk), 128, 0, s>>>(hist, K, n_bins, rho,
                                                                                                  part, rpart);
        VUP_CHECK_LAUNCH();
        k_sa_global_sum<<<(unsigned)ceil_div64(n_bins, 128), 128, 0, s>>>(part, rpart, nblk, n_bins, global);
        VUP_CHECK_LAUNCH();
    }
    return VUP_OK;
}
