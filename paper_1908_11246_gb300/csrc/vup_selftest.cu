// Self-test of the bounded-wait path: one CTA waits on an mbarrier that
// nothing arrives at, gives up after a fixed number of polls, records
// VUP_DSTAT_TIMEOUT in the grid's device status word and returns -- the same
// expiry path the tensor-core contraction and the histogram kernels take when
// a staged copy never lands, exercised without any fault.
#include "vup_internal.cuh"

namespace {

__global__ void k_wait_selftest(int *dstatus, uint32_t polls) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (uint32_t i = 0; i < polls; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a)
            : "memory");
        if (ok) return;
        __nanosleep(1000);
    }
    atomicCAS(dstatus, 0, VUP_DSTAT_TIMEOUT);
}

}  // namespace

extern "C" vup_status vup_selftest_wait(vup_grid g, uint32_t polls, vup_stream_t stream) {
    if (!g || polls < 1 || polls > (1u << 20)) return VUP_ERR_INVALID_ARG;
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(g->dstatus, polls);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}
