// Measured ceilings of the two CUDA-core resources the non-tensor kernels are
// bound by, for the roofline fractions of the measurement (not part of the
// method):
//   kind 0: FP32 fused multiply-add throughput (the plain FP32 contraction),
//           FLOP/s counting an FMA as two;
//   kind 1: shared-memory gathers of 512-byte rows (the segmented
//           histogram's access: a warp reads one 128-float row of a
//           shared-memory tile at a data-dependent row, 16 bytes per lane),
//           bytes/s through the SM's L1 data pipe.
// Both run on every SM at full occupancy for a fixed number of iterations
// and are timed with CUDA events on the caller's stream.
#include "vup_internal.cuh"

namespace {

constexpr int kPeakThreads = 256;

// Eight independent FMA chains per thread; the result feeds a store that a
// run never takes (the sum is finite), so nothing is optimised away.
__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(float *out, int iters, float b, float c) {
    float a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = (float)(threadIdx.x + q);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = fmaf(a[q], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += a[q];
    if (!(s == s) || s == 1.2345e38f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Rows of 32 float4 (512 bytes); each warp walks its own pseudo-random row
// sequence (a 32-bit LCG, the same on every lane, so a warp's 32 lanes read
// one contiguous row: four conflict-free wavefronts).
constexpr int kGatherRows = 128;  // 64 KB: three CTAs (24 warps) per SM
__global__ void __launch_bounds__(kPeakThreads) k_peak_gather(float *out, int iters) {
    extern __shared__ float4 tile[];  // [kGatherRows][32]
    for (int e = threadIdx.x; e < kGatherRows * 32; e += blockDim.x)
        tile[e] = make_float4((float)e, 1.f, 2.f, 3.f);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = 2654435761u * (uint32_t)(blockIdx.x * 64 + warp + 1);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            x = x * 1664525u + 1013904223u;
            const float4 v = tile[((x >> 24) & (kGatherRows - 1)) * 32 + lane];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    }
    const float s = acc.x + acc.y + acc.z + acc.w;
    if (!(s == s) || s == 1.2345e38f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" vup_status vup_measure_peak(int kind, vup_stream_t stream, double *value) {
    if (!value || kind < 0 || kind > 1) return VUP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = vup_num_sms();
    int per_sm = 0;
    const size_t smem = kind == 1 ? sizeof(float4) * kGatherRows * 32 : 0;
    if (kind == 1)
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_peak_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (kind == 0)
        VUP_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_ffma, kPeakThreads, 0));
    else
        VUP_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_gather, kPeakThreads, smem));
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    float *out = nullptr;
    VUP_CHECK_CUDA(vup_dev_malloc(&out, sizeof(float) * (size_t)blocks * kPeakThreads));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    const int iters = kind == 0 ? 4096 : 8192;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {  // the first pass warms up
        cudaEventRecord(e0, s);
        if (kind == 0)
            k_peak_ffma<<<blocks, kPeakThreads, 0, s>>>(out, iters, 0.999999f, 1e-7f);
        else
            k_peak_gather<<<blocks, kPeakThreads, smem, s>>>(out, iters);
        err = cudaGetLastError();
        cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    VUP_CHECK_CUDA(err);
    const double threads = (double)blocks * kPeakThreads;
    const double work = kind == 0 ? threads * iters * 16.0 * 8.0 * 2.0           // FLOP
                                  : threads / 32.0 * iters * 8.0 * 512.0;        // bytes
    *value = work / (ms * 1e-3);
    return VUP_OK;
}
