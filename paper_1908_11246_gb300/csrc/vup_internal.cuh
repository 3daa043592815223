// Internal declarations shared by the libvup CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "vup.h"

#define VUP_CHECK_CUDA(expr)                                                  \
    do {                                                                      \
        cudaError_t _e = (expr);                                              \
        if (_e != cudaSuccess) {                                              \
            vup_set_last_cuda_error(_e, #expr, __FILE__, __LINE__);           \
            return _e == cudaErrorMemoryAllocation ? VUP_ERR_OOM : VUP_ERR_CUDA; \
        }                                                                     \
    } while (0)

#define VUP_CHECK_LAUNCH() VUP_CHECK_CUDA(cudaGetLastError())

// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while the kernel before it in the stream is still running; it
// calls pdl_wait() before touching anything that kernel reads or writes
// (griddepcontrol.wait returns once the prerequisite grid has completed and
// its memory is visible; without a programmatic launch it returns at once).
// pdl_trigger() lets the next kernel be scheduled once every block of this
// one has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

void vup_set_last_cuda_error(cudaError_t e, const char *expr, const char *file, int line);

// Every device allocation of the library goes through vup_dev_malloc, which
// honours the allocation-failure hook of vup_debug_fail_alloc (tests of the
// out-of-memory paths) and otherwise calls cudaMalloc.
cudaError_t vup_dev_malloc_raw(void **p, size_t bytes);
template <typename T>
inline cudaError_t vup_dev_malloc(T **p, size_t bytes) {
    return vup_dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}

// hi + lo += x: TwoSum (Knuth) of hi and x, the rounding error kept in lo.
// FP32 sums of many terms are taken in short runs folded into such pairs,
// which keeps about FP32-squared accuracy over a long range.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

// Device status word codes (grid->dstatus[0]); the first non-zero code wins.
enum { VUP_DSTAT_OK = 0, VUP_DSTAT_EMPTY = 5, VUP_DSTAT_TIMEOUT = 6, VUP_DSTAT_BOUNDS = 7 };

// Device bounds checks of the debug build (-DVUP_DEBUG, libvup_debug.so):
// VUP_DBG_IN(i, n, dstatus) is true when 0 <= i < n; otherwise it records
// VUP_DSTAT_BOUNDS (returned by vup_sync as VUP_ERR_BOUNDS) and is false, and
// the caller skips or clamps the access instead of trapping.  In the release
// build it is the constant true and its arguments are not evaluated.
#ifdef VUP_DEBUG
__device__ __forceinline__ bool vup_dbg_in(uint64_t i, uint64_t n, int *dstatus) {
    if (i < n) return true;
    atomicCAS(dstatus, 0, VUP_DSTAT_BOUNDS);
    return false;
}
#define VUP_DBG_IN(i, n, dstatus) vup_dbg_in((uint64_t)(i), (uint64_t)(n), (dstatus))
#else
#define VUP_DBG_IN(i, n, dstatus) true
#endif

// Per-(k, axis) density constants written by the density-prep kernel.
//   Gaussian / truncated normal, index space: the midpoint index of mu is
//   c = (mu - lo) / h - 1/2 = n + f with integer n and f in [0, 1); the
//   density at midpoint a is exp(-((a - n) - f)^2 r^2 / 2) with r = h / sigma.
struct DensConst {
    int32_t n;      // integer part of the mean's index coordinate
    float f;        // fractional part
    float r;        // h / sigma
    int32_t kind;   // vup_density_kind
};

// Per-(k, axis) normalisation statistics (FP64).
struct DensStats {
    double invZ;    // 1 / sum_a g(a)
    double Eu;      // sum_a g u / sum_a g,   u = ((a - n) - f) r
    double Eu2;     // sum_a g u^2 / sum_a g
    double inv_sigma;
};

// Reference point and scale of the power tables: z = (y - c) / s with c the
// point of [ymin, ymax] nearest 0 (0 when the range holds it) and
// s = max |y - c| over the grid (1 when that is 0), so |z| <= 1.  With this c
// every |y| = |c| + s |z| (y and c have one sign), so the binomial
// re-expansion M_j = sum_m C(j, m) c^(j-m) s^m Mz_m of the raw moments keeps
// the error bound of the unshifted sum, while central moments are formed
// from Mz alone and lose nothing to a large common offset of y.
// The grid's device array holds {s, c, s_abs} with s_abs = max(|ymin|, |ymax|)
// (1 when 0), the unshifted scale of the supplied-weights paths.
__host__ __device__ inline void power_ref(double ymin, double ymax, double &c, double &s, double &s_abs) {
    c = ymin > 0.0 ? ymin : (ymax < 0.0 ? ymax : 0.0);
    const double a = fabs(ymin - c), b = fabs(ymax - c);
    s = a > b ? a : b;
    if (!(s > 0.0)) s = 1.0;
    const double m = fabs(ymin) > fabs(ymax) ? fabs(ymin) : fabs(ymax);
    s_abs = m > 0.0 ? m : 1.0;
}
// The power tables hold z^j 2^e (an exact power-of-two factor, removed again
// in FP64 by the finish): moments of outputs far below the grid's largest
// |y - c| keep FP32 / BF16 normal numbers (z^j down to 2^(-126-e)) instead of
// underflowing.  The largest contraction sum, sum_i g |z|^j 2^e with every
// factor g <= 1, stays below N 2^e; e = 120 - ceil(log2 N) leaves 2^6 of
// headroom under the FP32 range.
__host__ __device__ inline double power_factor(int64_t N) {
    int lg = 0;
    while (((int64_t)1 << lg) < N) ++lg;
    return ldexp(1.0, 120 - lg);
}
enum { kScaleS = 0, kScaleC = 1, kScaleAbs = 2, kScaleP = 3, kScaleSlots = 4 };

// Raw moments M_j = sum_i W y^j (j = 1..4) from mz[m-1] = sum_i W z^m
// (m = 1..4) and sum_i W = 1: M_j = sum_{m=0..j} C(j, m) c^(j-m) s^m Mz_m.
__host__ __device__ inline void raw_from_shifted(const double mz[4], double c, double s, double M[4]) {
    const double z[5] = {1.0, mz[0], mz[1], mz[2], mz[3]};
    double sp[5], cp[5];
    sp[0] = cp[0] = 1.0;
    for (int q = 1; q < 5; ++q) {
        sp[q] = sp[q - 1] * s;
        cp[q] = cp[q - 1] * c;
    }
    const double C[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
    for (int j = 1; j <= 4; ++j) {
        double v = 0.0;
        for (int m = 0; m <= j; ++m) v += C[j][m] * cp[j - m] * sp[m] * z[m];
        M[j - 1] = v;
    }
}

// Central moments from the shifted ones: mean = c + s Mz_1 and, for j >= 2,
// E[(y - mean)^j] = s^j sum_{m=0..j} C(j, m) (-Mz_1)^(j-m) Mz_m.
__host__ __device__ inline void central_from_shifted(const double mz[4], double c, double s, double out[4]) {
    const double z[5] = {1.0, mz[0], mz[1], mz[2], mz[3]};
    const double C[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
    const double a = -mz[0];
    double ap[5];
    ap[0] = 1.0;
    for (int q = 1; q < 5; ++q) ap[q] = ap[q - 1] * a;
    out[0] = c + s * mz[0];
    double sj = s;
    for (int j = 2; j <= 4; ++j) {
        sj *= s;
        double v = 0.0;
        for (int m = 0; m <= j; ++m) v += C[j][m] * ap[j - m] * z[m];
        out[j - 1] = sj * v;
    }
}

// Capacity-tracked device buffer.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};
vup_status devbuf_reserve(DevBuf &b, size_t bytes);
void devbuf_free(DevBuf &b);

// Layout of the contraction for one orientation of a grid.
//   red  : the reduction axes (flat index r), contiguous in y
//   rest : the remaining axes (flat index q), columns c = q * J + j
struct Orient {
    int red_axis0;      // first reduction axis
    int64_t R;          // reduction length
    int64_t R_pad;      // padded to a multiple of 64
    int64_t Q;          // number of rest points
    int64_t NC;         // Q * J
    int rest_axes[2];   // rest axes (up to 2), -1 if unused
    int64_t rest_n[2];  // their sizes (1 if unused); q = a_rest0 * rest_n[1] + a_rest1
    int n_rest_axes;
};

// Orientation indices: 0 = reduce over the last axis (every contraction of
// the forward moments, 2-D and 3-D), 1 = reduce over axis 0 (2-D, the IPSA
// derivatives of axis 1).
enum { kOrientLast = 0, kOrientFirst = 1, kNumOrient = 2 };

struct vup_grid_s {
    int device = 0;
    int ndim = 0;
    int64_t n[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    int64_t N = 0;

    // model outputs
    int have_model = 0;
    uint64_t model_gen = 0;        // bumped whenever the model (and its tables) are rebuilt
    int model_id = 0;              // built-in model of vup_eval_model (0: outputs set by the caller)
    double theta[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int B = 0, J = 0;
    double host_ext[3] = {0, 0, 1};  // ymin, ymax, s (filled lazily by vup_grid_info)

    double *y = nullptr;           // [N]
    double2 *axis_terms = nullptr; // [sum_d n_d] per-axis terms of separable built-in models
    unsigned long long *ext = nullptr;  // [2] ordered-bits min / max of y
    int32_t *bins = nullptr;       // [N]
    int32_t *perm = nullptr;       // [N] sorted position -> flat index
    int32_t *offsets = nullptr;    // [B_cap + 1]
    int32_t B_cap = 0;
    int natural_valid = 0;         // perm holds the stable sort by bin
    int layout_valid = 0;          // the histogram layout matches the current bins
    int layout_has_points = 0;     // ... and its key-sorted streams were built on request
    int range_ready = 0;           // ext holds the range of y (reduced by the model kernels)
    int bins_ready = 0;            // the model kernel also wrote the bins and the power-table scale
    // second stream for the layout build beside the density preparation
    // (forked from and joined back into the caller's stream)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_rec = nullptr;
    cudaStream_t side2 = nullptr;                       // the prefix-sum tiles beside the contraction
    cudaEvent_t ev_lay = nullptr, ev_dens = nullptr, ev_pre = nullptr, ev_mom = nullptr, ev_mfin = nullptr;

    // counting-sort scratch
    DevBuf sort_counts, scan_tmp, lay_tmp, rec_tmp;

    // histogram point streams.  Layout 0 gathers the last axis per point and
    // forms runs over the other axes; on 2-D grids layout 1 swaps the roles
    // (points ordered by (bin, a1, a0)).  The device picks the layout with
    // fewer intervals (hist_sel[0], counted before sorting) and builds only
    // that one: the arrays live in hl[0], hl[1] holds layout 1's geometry and
    // aliases them.
    struct HistLayout {
        int last_axis = -1;            // axis gathered per point
        int64_t n_last = 0;
        int P = 1;                     // parts of the gathered axis (shared-memory tiles)
        int64_t part_rows = 0;         // gathered-axis rows per part
        int32_t *keys = nullptr;       // sort key of the layout's flat index: part * B + bin
        int32_t *keys_own = nullptr;   // [N] key storage
        int32_t *koff = nullptr;       // [P * B + 1] key offsets in the sorted stream
        int2 *key_chunks = nullptr;    // [P * B] first and last chunk of each key's points (-1 if empty)
        int32_t koff_cap = 0;
        int32_t *perm = nullptr;       // [N] sorted position -> layout flat index
        uint32_t *hpt = nullptr;       // [N + 512] packed per-point word
        int32_t *run_start = nullptr;  // [N + 1]
        int32_t *run_rest = nullptr;   // [N]
        int32_t *run_bin = nullptr;    // [N]
        int32_t *n_runs = nullptr;     // [1] device
        int32_t *chunk_pt = nullptr;   // [P * n_chunks + 1] chunk start (point index)
        int32_t *chunk_run = nullptr;  // [P * n_chunks + 1] chunk start (run index)
        int32_t *chunk_bin = nullptr;  // [P * n_chunks * 2] first / last key of each chunk
        // interval stream: maximal stretches of a run whose gathered-axis rows
        // are consecutive; uint2 (first row << shift, (last row + 1) << shift |
        // run-end / key-end flags | rest code of interval + 4)
        uint2 *ipt = nullptr;          // [N + 128]
        int32_t *iv_rest = nullptr;    // [N] rest index of each interval
        int32_t *n_iv = nullptr;       // [1] device
        int32_t *chunk_iv = nullptr;   // [P * n_chunks + 1] chunk start (interval index)
        // record stream: one record per (line, group of 4 consecutive bins,
        // monotone stretch): two uint4 per record, sorted by (part, group, line)
        DevBuf rec;                    // [n_rec + 16][2] uint4
        DevBuf rec_rest;               // [n_rec] rest index of each record
        DevBuf rec_goff;               // [n_groups + 2] first record of each group
        DevBuf rec_gch;                // [n_groups] int2: first / last chunk holding the group (-1 if empty)
        int32_t *rec_chunk = nullptr;  // [P * n_chunks_rec + 1] chunk start (record index)
        int32_t *rec_chunk_grp = nullptr;  // [P * n_chunks_rec * 2] first / last group of each chunk
        int32_t *n_rec = nullptr;      // [1] device
    } hl[2];
    int hist_P = 1;                // max parts over layouts (scratch sizing)
    int n_layouts = 1;
    int32_t *hist_sel = nullptr;   // [4] device: chosen layout, 1 = interval stream, intervals of layouts 0 / 1
    int hist_force = -1;           // -1 auto, 0 points only, 1 intervals only
    int32_t n_chunks = 0;
    int32_t n_chunks_rec = 0;      // record chunks per part (records are several times fewer than points)

    // power tables per orientation (kOrient*)
    Orient orient[kNumOrient];
    int have_tab[kNumOrient][3] = {};               // [orient][0: fp32, 1: bf16, 2: tf32]
    float *zs[kNumOrient] = {};                      // SIMT layout [R][NC]
    __nv_bfloat16 *zt_hi[kNumOrient] = {};           // tensor layout [NC][R_pad]
    __nv_bfloat16 *zt_lo[kNumOrient] = {};
    float *ztf_hi[kNumOrient] = {};                  // tensor layout [NC][R_pad], TF32 values
    float *ztf_lo[kNumOrient] = {};
    double *ydev_scale = nullptr;  // [1] s on device

    // per-K scratch (density constants, factor tables, partials)
    int64_t K_cap = 0;
    DevBuf dconst, dstats, dpart, ftab, atab_hi, atab_lo, partials, hist_part, hist_direct, ipsa_part;
    DevBuf hist_prefix;  // prefix-sum tiles of the gathered axis [P][K_pad / 128][rows + 1][128]
    DevBuf atf_hi, atf_lo;         // TF32 split of the A operand [K_pad][R_pad]

    // supplied-weights path: the grid points in blocks of 256, each block's
    // points sorted by bin (word: local index | bin << 8), their powers of
    // z = y / s_abs in that order, and every block's split into eight warp
    // slices at bin boundaries; built for model generation wsort_gen
    DevBuf wsort_pt, wsort_z, wsort_fix;
    uint64_t wsort_gen = ~0ull;
    int weights_form = -1;         // supplied-W form: -1 auto, 0 sorted walk, 1 row per lane, 2 general

    int *dstatus = nullptr;        // [1] device status word
};

// ---- kernels / launchers implemented in the .cu files -------------------
vup_status vup_launch_model_at(vup_grid g, int64_t K, const double *x, double *y, cudaStream_t s);
vup_status vup_launch_model_eval(vup_grid g, int model_id, const double *theta,
                                 cudaStream_t s);
vup_status vup_launch_grid_finish(vup_grid g, cudaStream_t s);  // range, bins (1-D: the sorted order)
vup_status vup_pick_hist_layout(vup_grid g, cudaStream_t s);
// Histogram layout (2-D / 3-D): built on first use after a model evaluation.
// points_needed: the key-sorted point stream is built whatever the device
// would choose (callers that walk it: posterior means).
// records_done (optional) is recorded on s once the record stream is complete
// (the key-sorted streams follow); layout_picked (optional) once the layout
// (hist_sel[0]) is chosen.
vup_status vup_build_layout(vup_grid g, cudaStream_t s, bool points_needed = false,
                            cudaEvent_t records_done = nullptr, cudaEvent_t layout_picked = nullptr);
vup_status vup_ensure_layout(vup_grid g, cudaStream_t s, bool points_needed = false);
// every layout's part tile fits the shared-memory histogram kernels
bool vup_hist_tile_fits(vup_grid g);
// the 3-D point stream stages both rest-axis factor tables in shared memory
// (and its run-end words then carry the next run's rest code)
bool vup_hist_rest_staged(const vup_grid_s *g);
vup_status vup_build_tables(vup_grid g, int orient, int bf16, cudaStream_t s);
vup_status vup_natural_sort(vup_grid g, cudaStream_t s);

// Density factors and normalisers; the A-operand split tables of the
// orientations in the mask (BF16 into atab_*, or TF32 into atf_* when tf32);
// stats: also E[u] and E[u^2] per (k, d) (the IPSA derivatives need them).
vup_status vup_density_prep(vup_grid g, const vup_densities *d, int need_bf16_orient_mask,
                            cudaStream_t s, bool tf32 = false, bool stats = false);
vup_status vup_moments_simt(vup_grid g, int64_t K, int orient, int n_out, float *part, cudaStream_t s);
// Tensor-core contraction; kind 0 = BF16 operands, 1 = TF32 operands;
// terms = 3 split products or 1 (hi only).
vup_status vup_moments_tc(vup_grid g, int64_t K, int orient, int n_out, float *part, cudaStream_t s,
                          int kind = 0, int terms = 3);
// FP64 finish of the contraction partials [n_col_tiles][K_pad][4] at `part`
// (NULL: the grid's moment partials)
vup_status vup_moments_finish(vup_grid g, int64_t K, int n_col_tiles, double *raw,
                              double *central, cudaStream_t s, const float *part = nullptr);
// Segmented histogram of the K densities; `ftab` replaces the grid's factor
// tables when not null (same layout), e.g. tables weighted by a coordinate.
// points_only: walk the point stream even where the interval stream was
// chosen (sums that must keep their relative accuracy in low-mass bins, as
// the numerators and denominators of ratios do).
// keys_ready (optional): an event the point and interval kernels (and the
// finish) wait for; the record-stream kernel is launched before that wait.
// prefix_ready: vup_hist_prefix already wrote the prefix-sum tiles for
// these densities (on a stream s has waited for).
vup_status vup_hist_fused(vup_grid g, int64_t K, float *hist, cudaStream_t s, const float *ftab = nullptr,
                          bool points_only = false, cudaEvent_t keys_ready = nullptr, bool prefix_ready = false);
// The interval and record streams' prefix-sum tiles of the chosen layout for K
// densities (after their preparation and the layout choice), whichever
// stream the device picks later; false when the grid's histogram does not
// run the shared-memory kernels (nothing launched).
bool vup_hist_prefix(vup_grid g, int64_t K, cudaStream_t s);
vup_status vup_propagate_1d(vup_grid g, const vup_densities *d, double *raw, double *central,
                            float *hist, cudaStream_t s);
vup_status vup_ipsa_1d(vup_grid g, const vup_densities *d, const double *grad, float *dmu,
                       float *dsg, cudaStream_t s);
vup_status vup_ipsa_finish(vup_grid g, int64_t K, int n_tiles0, int n_tiles1,
                           const double *grad, float *dmu, float *dsg, cudaStream_t s);
vup_status vup_weights_path(vup_grid g, int64_t K, const float *W, double *raw, float *hist,
                            cudaStream_t s);

int vup_num_sms();
// Orientation of the forward tensor-core contraction: the last axis is the
// reduction (3-D grids apply both rest axes' factors in the epilogue).
inline int vup_tc_orient(const vup_grid_s *) { return kOrientLast; }
bool vup_profiling();
vup_status vup_check_dens(vup_grid g, const vup_densities *d);
vup_status vup_reserve_k(vup_grid g, int64_t K, bool bf16, bool ipsa, bool tf32 = false);

// Batched stages over many 2-D instances.  Each *_plan builds host-side work
// lists and uploads them into device memory it owns (synchronous; never call
// during stream capture); each *_batched launch is stream-ordered and
// capturable; *_plan_free releases a plan.
vup_status vup_density_reserve(vup_grid g, int64_t K);
vup_status vup_density_plan(int n, const vup_grid *gs, const vup_densities *ds, bool bf16, void **plan);
vup_status vup_density_batched(void *plan, cudaStream_t s);
void vup_density_plan_free(void *plan);
int64_t vup_tc_col_tiles_bn(const Orient &o, int bn);
int vup_tc_bn_for(const Orient &o, int bn_cap);
vup_status vup_tc_plan(int n, const vup_grid *gs, const int64_t *Ks, const int *bns, float *const *parts,
                       void **plan);
vup_status vup_tc_batched(void *plan, int *dstatus, cudaStream_t s);
void vup_tc_plan_free(void *plan);
vup_status vup_simt_plan(int n, const vup_grid *gs, const int64_t *Ks, float *const *parts, void **plan);
vup_status vup_simt_batched(void *plan, cudaStream_t s);
void vup_simt_plan_free(void *plan);
vup_status vup_finish_plan(int n, const vup_grid *gs, const int64_t *Ks, const int64_t *n_cts,
                           float *const *parts, double *const *raws, double *const *centrals, void **plan);
vup_status vup_finish_batched(void *plan, cudaStream_t s);
void vup_finish_plan_free(void *plan);
bool vup_hist_batchable(vup_grid g);
vup_status vup_hist_plan(int n, const vup_grid *gs, const int64_t *Ks, float *const *hists, void **plan);
vup_status vup_hist_batched(void *plan, cudaStream_t s);
void vup_hist_plan_free(void *plan);

// Per-kernel timing scope (active only while vup_profile(1) is in effect):
// records a CUDA event pair on `s` around the launches made in its lifetime.
struct ProfScope {
    ProfScope(const char *name, cudaStream_t s, int launches = 1);
    ~ProfScope();
    const char *name;
    cudaStream_t stream;
    int launches;
    int slot;
};
#define VUP_PROF_CAT2(a, b) a##b
#define VUP_PROF_CAT(a, b) VUP_PROF_CAT2(a, b)
#define VUP_PROF(name, s, n) ProfScope VUP_PROF_CAT(_vup_prof_, __LINE__)(name, s, n)

// Column-tile counts used by the contraction kernels (for the finish step).
int64_t vup_simt_col_tiles(const Orient &o);
// partial columns of a contraction of K densities, and the most any K can need
int64_t vup_tc_col_tiles(const Orient &o, int64_t K);
int64_t vup_tc_col_tiles_max(const Orient &o);

// Scratch sizes per K row.
size_t vup_ftab_floats(const vup_grid g);   // sum_d n[d] floats per k

static inline int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }
