// Supplied-weights propagation that allocates no device memory.
//
// Same arithmetic as vup_propagate_weights (moments of the power table and
// histograms of every row of a caller-supplied weight matrix), but its
// per-call scratch -- the per-split partial moments and partial histograms --
// lives in one file-scope device array of fixed size instead of memory the
// library allocates on first use.  It exists for callers that cannot call
// cudaMalloc once their hot loop runs: hosts with a fixed device-memory
// budget, allocators that forbid growth after start-up, or code embedded in
// a runtime that owns the device heap.
#include "vup_internal.cuh"

#include <algorithm>
#include <mutex>

namespace {

constexpr int kThreads = 256;
constexpr size_t kScratchBytes = VUP_STATIC_SCRATCH_BYTES;

// Shared by every call on a device; holds [n_split][K][4] partial moments
// (double) followed by [n_split][K][B] partial histograms (float).  Every
// element a call reads was written by the same call, so nothing needs
// clearing between calls.
static __device__ __align__(256) unsigned char vup_static_scratch[kScratchBytes];

template <int RB>
__global__ void __launch_bounds__(kThreads) k_weights_static(const float *__restrict__ W, int64_t K, int64_t N,
                                                             const double *__restrict__ y,
                                                             const double *__restrict__ scale,
                                                             const int32_t *__restrict__ bins, int B,
                                                             int64_t n_split, double *__restrict__ mpart,
                                                             float *__restrict__ hpart) {
    extern __shared__ float sh[];  // [RB][B]
    __shared__ double red[RB][4][kThreads / 32];
    const int64_t split = blockIdx.x;
    const int64_t k0 = (int64_t)blockIdx.y * RB;
    for (int e = threadIdx.x; e < RB * B; e += blockDim.x) sh[e] = 0.f;
    __syncthreads();
    const double s = scale[kScaleAbs];
    const int64_t per = (N + n_split - 1) / n_split;
    const int64_t i0 = split * per, i1 = min(N, i0 + per);
    float m[RB][4], ml[RB][4];  // TwoSum pairs (two_sum_acc)
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int j = 0; j < 4; ++j) m[r][j] = ml[r][j] = 0.f;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const float p = (float)(y[i] / s);
        const int bq = bins[i];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            if (k0 + r >= K) break;
            const float w = W[(k0 + r) * N + i];
            float t = w * p;
            two_sum_acc(m[r][0], ml[r][0], t);
            t *= p;
            two_sum_acc(m[r][1], ml[r][1], t);
            t *= p;
            two_sum_acc(m[r][2], ml[r][2], t);
            t *= p;
            two_sum_acc(m[r][3], ml[r][3], t);
            atomicAdd(&sh[r * B + bq], w);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double v = (double)m[r][j] + (double)ml[r][j];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[r][j][warp] = v;
        }
    __syncthreads();
    if (threadIdx.x < RB * 4) {
        const int r = threadIdx.x >> 2, j = threadIdx.x & 3;
        double v = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) v += red[r][j][w];
        if (k0 + r < K) mpart[(split * K + k0 + r) * 4 + j] = v;
    }
    for (int e = threadIdx.x; e < RB * B; e += blockDim.x) {
        const int r = e / B, b = e - r * B;
        if (k0 + r < K) hpart[(split * K + k0 + r) * B + b] = sh[e];
    }
}

__global__ void k_weights_static_finish(const double *__restrict__ mpart, const float *__restrict__ hpart,
                                        int64_t n_split, int64_t K, int B, int J, const double *__restrict__ scale,
                                        double *__restrict__ raw, float *__restrict__ hist) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (hist && e < K * B) {
        float s = 0.f;
        for (int64_t q = 0; q < n_split; ++q) s += hpart[q * K * B + e];
        hist[e] = s;
    }
    if (raw && e < K * J) {
        const int64_t k = e / J;
        const int j = (int)(e - k * J);
        double s = 0.0;
        for (int64_t q = 0; q < n_split; ++q) s += mpart[(q * K + k) * 4 + j];
        double sp = scale[kScaleAbs];
        for (int q = 0; q < j; ++q) sp *= scale[kScaleAbs];
        raw[e] = s * sp;
    }
}

// Device address of the scratch array, resolved once per device.
std::mutex g_scratch_mu;
void *g_scratch_addr[64];

vup_status scratch_address(void **out) {
    int dev = 0;
    VUP_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return VUP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        VUP_CHECK_CUDA(cudaGetSymbolAddress(&p, vup_static_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return VUP_OK;
}

}  // namespace

extern "C" vup_status vup_propagate_weights_noalloc(vup_grid g, int64_t K, const float *W, double *moments_raw,
                                                    float *hist, vup_stream_t stream) {
    if (!g || !W || K < 1) return VUP_ERR_INVALID_ARG;
    if (!g->have_model) return VUP_ERR_STATE;
    const int64_t N = g->N;
    const int B = g->B;
    const int RB = B <= 3072 ? 8 : (B <= 6144 ? 4 : 2);
    // bytes one split needs: K rows of 4 partial moments and B partial bins
    const size_t per_split = (size_t)K * (4 * sizeof(double) + (size_t)B * sizeof(float));
    if (per_split > kScratchBytes) return VUP_ERR_INVALID_ARG;
    void *scratch = nullptr;
    vup_status st = scratch_address(&scratch);
    if (st != VUP_OK) return st;
    const int64_t rows = ceil_div64(K, RB);
    if (rows > 65535) return VUP_ERR_UNSUPPORTED;  // one CTA row per RB densities
    int64_t n_split = std::max<int64_t>(1, (int64_t)vup_num_sms() * 8 / std::max<int64_t>(rows, 1));
    n_split = std::min<int64_t>(n_split, std::max<int64_t>(1, N / 4096));
    n_split = std::min<int64_t>(n_split, (int64_t)(kScratchBytes / per_split));
    double *mpart = reinterpret_cast<double *>(scratch);
    float *hpart = reinterpret_cast<float *>(mpart + (size_t)4 * K * n_split);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = sizeof(float) * (size_t)RB * B;
    dim3 grd((unsigned)n_split, (unsigned)rows);
    if (RB == 8) {
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_weights_static<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
        k_weights_static<8><<<grd, kThreads, smem, s>>>(W, K, N, g->y, g->ydev_scale, g->bins, B, n_split, mpart, hpart);
    } else if (RB == 4) {
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_weights_static<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
        k_weights_static<4><<<grd, kThreads, smem, s>>>(W, K, N, g->y, g->ydev_scale, g->bins, B, n_split, mpart, hpart);
    } else {
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_weights_static<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
        k_weights_static<2><<<grd, kThreads, smem, s>>>(W, K, N, g->y, g->ydev_scale, g->bins, B, n_split, mpart, hpart);
    }
    VUP_CHECK_LAUNCH();
    const int64_t tot = std::max<int64_t>(K * B, K * g->J);
    k_weights_static_finish<<<(unsigned)ceil_div64(tot, 256), 256, 0, s>>>(mpart, hpart, n_split, K, B, g->J,
                                                                           g->ydev_scale, moments_raw, hist);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}
