// Bayes-inverted model matrix (Sec. 3: the inverted model matrix built from
// Bayes' theorem maps an output bin back to the input points that reach it,
// each with posterior probability W[k,i] / H[k,b]), applied to the input
// coordinates: the posterior mean of every input axis per output bin,
//   post[k][b][d] = sum_{i in b} W[k,i] x_{d,i} / H[k,b].
// The numerators are histograms of the densities with one axis' factor
// table multiplied by that axis' coordinates, so each axis is one more pass
// of the segmented histogram kernel; W is never formed.
#include "vup_internal.cuh"

namespace {

// xtab rows of axis d (rows row0 .. row0 + n - 1) = ftab rows times x_{d,a}.
__global__ void k_weight_axis(const float *__restrict__ ftab, float *__restrict__ xtab, int64_t row0, int64_t n,
                              int64_t K_pad, double lo, double h) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * K_pad) return;
    const int64_t a = e / K_pad;
    const double x = __dadd_rn(lo, __dmul_rn(__dadd_rn((double)a, 0.5), h));
    xtab[row0 * K_pad + e] = ftab[row0 * K_pad + e] * (float)x;
}

// post[k][b][d] = hx[d][k][b] / hist[k][b] (0 where the bin has no mass).
__global__ void k_posterior_finish(const float *__restrict__ hist, const float *__restrict__ hx, int64_t K, int B,
                                   int nd, float *__restrict__ post) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= K * B) return;
    const float h = hist[e];
    for (int d = 0; d < nd; ++d) post[e * nd + d] = h > 0.f ? hx[(int64_t)d * K * B + e] / h : 0.f;
}

DevBuf g_xtab, g_hx, g_hist;  // process-wide scratch of this path

}  // namespace

extern "C" vup_status vup_posterior_means(vup_grid g, const vup_densities *d, float *hist, float *post,
                                          vup_stream_t stream) {
    if (!g || !post) return VUP_ERR_INVALID_ARG;
    vup_status st = vup_check_dens(g, d);
    if (st != VUP_OK) return st;
    if (!g->have_model) return VUP_ERR_STATE;
    if (g->ndim < 2) return VUP_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t K = d->K, K_pad = ceil_div64(K, 128) * 128;
    const int B = g->B, nd = g->ndim;
    const size_t tab = (size_t)K_pad * vup_ftab_floats(g);
    if ((st = vup_reserve_k(g, K, false, false)) != VUP_OK) return st;
    if ((st = devbuf_reserve(g_xtab, sizeof(float) * tab)) != VUP_OK) return st;
    if ((st = devbuf_reserve(g_hx, sizeof(float) * (size_t)nd * K * B)) != VUP_OK) return st;
    if (!hist) {
        if ((st = devbuf_reserve(g_hist, sizeof(float) * (size_t)K * B)) != VUP_OK) return st;
        hist = (float *)g_hist.p;
    }
    if ((st = vup_ensure_layout(g, s, true)) != VUP_OK) return st;  // the ratios walk the point stream
    if ((st = vup_density_prep(g, d, 0, s)) != VUP_OK) return st;
    // point stream: the ratios need the relative accuracy of low-mass bins,
    // which differences of prefix sums (interval stream) do not keep
    if ((st = vup_hist_fused(g, K, hist, s, nullptr, true)) != VUP_OK) return st;
    float *xtab = (float *)g_xtab.p;
    const float *ftab = (const float *)g->ftab.p;
    VUP_CHECK_CUDA(cudaMemcpyAsync(xtab, ftab, sizeof(float) * tab, cudaMemcpyDeviceToDevice, s));
    int64_t row0 = 0;
    for (int ax = 0; ax < nd; ++ax) {
        const int64_t n = g->n[ax];
        const double h = (g->hi[ax] - g->lo[ax]) / (double)n;
        {
            VUP_PROF("posterior_axis_weights", s, 1);
            k_weight_axis<<<(unsigned)ceil_div64(n * K_pad, 256), 256, 0, s>>>(ftab, xtab, row0, n, K_pad, g->lo[ax], h);
            VUP_CHECK_LAUNCH();
        }
        if ((st = vup_hist_fused(g, K, (float *)g_hx.p + (size_t)ax * K * B, s, xtab, true)) != VUP_OK) return st;
        VUP_CHECK_CUDA(cudaMemcpyAsync(xtab + row0 * K_pad, ftab + row0 * K_pad, sizeof(float) * n * K_pad,
                                       cudaMemcpyDeviceToDevice, s));
        row0 += n;
    }
    VUP_PROF("posterior_finish", s, 1);
    k_posterior_finish<<<(unsigned)ceil_div64(K * B, 256), 256, 0, s>>>(hist, (const float *)g_hx.p, K, B, nd, post);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}
