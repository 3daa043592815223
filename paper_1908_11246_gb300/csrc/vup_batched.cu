// Batched uneven propagation -- placeholder until the persistent kernel lands.
#include "vup_internal.cuh"

extern "C" vup_status vup_propagate_batched(int n_inst, const vup_grid *g, const vup_densities *d,
                                            vup_precision precision, double *const *moments_raw,
                                            float *const *hist, vup_stream_t stream) {
    (void)n_inst; (void)g; (void)d; (void)precision; (void)moments_raw; (void)hist; (void)stream;
    return VUP_ERR_UNSUPPORTED;
}
