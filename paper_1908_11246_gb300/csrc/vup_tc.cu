// Tensor-core (tcgen05) moment contraction -- placeholder until the kernel lands.
#include "vup_internal.cuh"

int64_t vup_tc_col_tiles(const Orient &o) { return ceil_div64(o.NC, 256); }

vup_status vup_moments_tc(vup_grid, int64_t, int, int, float *, cudaStream_t) { return VUP_ERR_UNSUPPORTED; }
