/*
 * vup.h -- C ABI of libvup.so, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of Vectorized Uncertainty Propagation (VUP) and
 * Input Probability Sensitivity Analysis (IPSA), arXiv 1908.11246.
 *
 * The calls follow the paper's statement of the problem:
 *   1. a uniform grid of midpoints over the input domain (Sec. 3, composite
 *      midpoint rule; Algorithm "VUP - Single probability", first step);
 *   2. the model evaluated once on that grid, and the model matrix built
 *      from it (Eq. 5 and Eq. MUP: a one-hot matrix that sorts every grid
 *      point into its output bin);
 *   3. K input densities pushed through that single model matrix at once
 *      (Eq. VUP), giving per-density output histograms (Eq. 4) and moments;
 *   4. IPSA sensitivities of those moments to each density's location and
 *      width (Sec. 5.2).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Grid: ndim in {1,2,3} axes; axis d has n[d] midpoints
 *   x_{d,a} = lo[d] + (a + 1/2) (hi[d] - lo[d]) / n[d].  The flat index is
 *   row-major with axis 0 slowest.  N = prod n[d].
 * - Densities are products over axes of one-dimensional densities
 *   (Gaussian as in Eq. gaussh, uniform, truncated normal), evaluated at the
 *   midpoints and normalised over the grid, i.e. hard-truncated at the domain
 *   boundary and renormalised (Sec. 5.3).
 * - Output bins: B equal-width bins over [min y, max y], half-open, the last
 *   closed: bin = min(floor((y - ymin) / (ymax - ymin) * B), B - 1), all in
 *   IEEE double with correctly rounded operations (Eq. 4).
 * - Moments: raw[k][j-1] = sum_i W[k,i] y_i^j and central[k][0] = mean,
 *   central[k][j-1] = E[(y - mean)^j] (j = 2..J), J = n_moments <= 4.
 * - Pointers documented as "device" must point to memory of the current CUDA
 *   device; "host" pointers are read during the call and not retained.
 *   The caller owns every buffer it passes; the grid owns its internals.
 * - Every call returns a vup_status.  Argument errors are detected on the
 *   host before any work is queued and leave all outputs untouched.
 *   Conditions detected on the device (a density with no grid point in its
 *   support, a bounded device-side wait that expired, and in the debug build
 *   a failed bounds check) are recorded in the grid's device status word and
 *   returned by vup_sync().  No call exits, aborts or traps.
 * - Debug build: libvup_debug.so exports the same ABI, compiled with
 *   VUP_DEBUG: the histogram walks and the supplied-weights walk check every
 *   row, column and histogram index they read from a layout or a sorted word
 *   against the array it addresses, record VUP_ERR_BOUNDS and skip the access
 *   (no trap).  The Python binding loads it when VUP_DEBUG=1.
 * - Stream-ordered calls enqueue work on `stream` and return without
 *   synchronising.  A grid must not be used from two streams concurrently.
 */
#ifndef VUP_H
#define VUP_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *vup_stream_t; /* == cudaStream_t; NULL = legacy default stream */

typedef struct vup_grid_s *vup_grid;

typedef enum {
    VUP_OK = 0,
    VUP_ERR_INVALID_ARG = 1,   /* bad shape, null required pointer, out-of-range value */
    VUP_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    VUP_ERR_OOM = 3,           /* device allocation failed */
    VUP_ERR_STATE = 4,         /* grid has no model outputs yet (call vup_eval_model first) */
    VUP_ERR_EMPTY_SUPPORT = 5, /* some density holds no grid point in its support */
    VUP_ERR_TIMEOUT = 6,       /* a bounded device-side wait expired; results are invalid */
    VUP_ERR_UNSUPPORTED = 7,   /* valid request this build does not implement */
    VUP_ERR_BOUNDS = 8         /* debug build (libvup_debug.so, compiled with VUP_DEBUG) only: a device
                                  bounds check on an index read from a layout or a sorted word failed;
                                  the access was skipped and the results are invalid */
} vup_status;

typedef enum { VUP_GAUSS = 0, VUP_UNIFORM = 1, VUP_TRUNCNORM = 2 } vup_density_kind;

typedef enum {
    VUP_FP64 = 0,   /* 1-D grids only: every step in double precision            */
    VUP_FP32 = 1,   /* plain FP32 CUDA-core contraction, FP64 final reduction     */
    VUP_BF16X3 = 2, /* tcgen05 tensor cores, 3 split BF16 products, FP32 accumulate */
    VUP_TF32 = 3,   /* tcgen05 tensor cores, one TF32 product (~1e-3: comparison only) */
    VUP_TF32X3 = 4  /* tcgen05 tensor cores, 3 split TF32 products, FP32 accumulate */
} vup_precision;

/* Built-in models (model_id of vup_eval_model).  theta is a host array. */
typedef enum {
    VUP_MODEL_SIN_QUAD_1D = 1,     /* y = t0 sin x + t1 x^2                         (1 axis) */
    VUP_MODEL_SIN_SIN2_2D = 2,     /* y = t0 sin x1 + t1 sin^2 x2    (Sec. 4.1)     (2 axes) */
    VUP_MODEL_MIXED_3D = 3,        /* y = sin x1 + t0 sin^2 x2 + t1 x3^4 sin x1     (3 axes) */
    VUP_MODEL_OSCILLATOR_2D = 4,   /* y = exp(-x2 x1 t0) cos(x1 sqrt(1 - x2^2) t0)  (2 axes) */
    VUP_MODEL_IPSA_EXAMPLE_2D = 5, /* y = x1^2 + 5 sin(3 x1) + x2    (Sec. 5.3)     (2 axes) */
    VUP_MODEL_POLY = 6             /* y = t0 + sum_d (t[1+2d] x_d + t[2+2d] x_d^2)  (1-3 axes) */
} vup_model_id;

/*
 * Densities, structure of arrays with element [k * ndim + d], for
 * 1 <= K <= VUP_MAX_DENSITIES (else the calls taking them return
 * VUP_ERR_INVALID_ARG; so does K < 1 in vup_propagate_weights).  All
 * pointers are device pointers owned by the caller and must stay valid until
 * the queued work has run.
 *   kind  : uint8 vup_density_kind per (k, d)
 *   mu    : Gaussian / truncated-normal mean; uniform centre
 *   sigma : Gaussian / truncated-normal standard deviation (> 0);
 *           uniform full width (> 0), support |x - mu| <= sigma / 2
 *   lo,hi : truncated-normal absolute bounds (support lo <= x <= hi);
 *           may be NULL when no axis is truncated normal
 */
typedef struct {
    int64_t K;
    int32_t ndim;
    const uint8_t *kind;
    const double *mu;
    const double *sigma;
    const double *lo;
    const double *hi;
} vup_densities;

/* Limits of this build. */
#define VUP_MAX_BINS 8192
#define VUP_MAX_MOMENTS 4
#define VUP_MAX_AXIS_POINTS 32767
#define VUP_MAX_DENSITIES (1 << 22)   /* K per call (larger K: split the call) */

/*
 * Create a grid (Sec. 3 uniform midpoint grid).  n, lo, hi: host arrays of
 * length ndim; 1 <= n[d] <= VUP_MAX_AXIS_POINTS, lo[d] < hi[d], finite.
 * Allocates device memory synchronously on the current device.
 * *out receives the handle; release it with vup_grid_destroy.
 */
vup_status vup_grid_create(int ndim, const int64_t *n, const double *lo, const double *hi,
                           vup_grid *out);

/* Free every device allocation the grid owns (synchronises the device). */
vup_status vup_grid_destroy(vup_grid g);

/*
 * Evaluate a built-in model on the grid and build the model matrix (Sec. 2
 * model function; Algorithm "VUP - Single probability" steps 1-2 and the
 * sparse model-matrix construction; Eq. MUP):
 *   y_i = M(x_i; theta) in FP64, [min y, max y], per-point bin ids; on 1-D
 *   grids a stable counting sort of the grid points by bin (the CSR form of
 *   the one-hot model matrix), on 2-D / 3-D grids the sorted histogram
 *   layout is built by the first vup_propagate that needs it; the power
 *   tables z^j, j = 1..n_moments, of z = (y - c) / s (c the point of
 *   [min y, max y] nearest 0, s = max |y - c|: raw moments are re-expanded
 *   from them in FP64, central moments formed from them directly) are
 *   built on first use, except that a separable built-in model on a 2-D /
 *   3-D grid writes the tensor-core contraction's split BF16 table here: its
 *   values, range, bins and that table come from one cooperative launch,
 *   whose blocks meet at a bounded grid barrier (an expired wait is reported
 *   by vup_sync as VUP_ERR_TIMEOUT).
 * theta: host array of n_theta doubles (n_theta <= 8).
 * 1 <= n_bins <= VUP_MAX_BINS, 1 <= n_moments <= VUP_MAX_MOMENTS.
 * Model values must be finite.
 */
vup_status vup_eval_model(vup_grid g, int model_id, const double *theta, int n_theta,
                          int n_bins, int n_moments, vup_stream_t stream);

/*
 * Same as vup_eval_model but with model values supplied by the caller:
 * y_dev is a device array of N finite doubles in flat grid order (a user
 * model evaluated elsewhere).  It is copied; the caller keeps ownership.
 */
vup_status vup_set_outputs(vup_grid g, const double *y_dev, int n_bins, int n_moments,
                           vup_stream_t stream);

/*
 * Push K densities through the grid's model matrix at once (Eq. VUP):
 *   moments_raw     [K][J] double, device, or NULL
 *   moments_central [K][J] double, device, or NULL
 *   hist            [K][B] float,  device, or NULL   (Eq. 4 output probabilities)
 * J and B are the values given to vup_eval_model.  precision selects the
 * contraction: VUP_FP64 requires ndim == 1; 1-D grids run in FP64 when
 * VUP_FP64 or VUP_FP32 is requested; the tensor-core kinds (VUP_BF16X3,
 * VUP_TF32, VUP_TF32X3) need ndim >= 2.  W[k, i] is generated on the fly
 * and never stored.  The first call with a larger K than before allocates
 * per-K scratch (not capturable in a CUDA graph), and the first TF32 call on
 * a grid builds its TF32 power tables; later calls allocate nothing.
 * When the histogram's layout is (re)built by the call (the first call after
 * vup_eval_model or vup_set_outputs), the grid runs parts of the work on two
 * streams of its own (the layout beside the density preparation and the
 * contraction; the prefix sums and the FP64 moments finish beside those) that
 * fork from and join back into `stream`: every result is complete, in stream
 * order, once the work queued on `stream` by this call is.  The grid creates
 * those streams and their events on first use.
 */
vup_status vup_propagate(vup_grid g, const vup_densities *d, vup_precision precision,
                         double *moments_raw, double *moments_central, float *hist,
                         vup_stream_t stream);

/*
 * Supplied-weights variant (Eq. VUP with the input probability matrix given
 * explicitly, as the paper materialises it): W is a device [K][N] float
 * array of per-grid-point weights (used as given, not renormalised).
 *   moments_raw [K][J] double (device, or NULL), hist [K][B] float (device, or NULL).
 * K <= 65535 x (2 .. 32) depending on B (VUP_ERR_UNSUPPORTED beyond); the
 * memory of W bounds K long before that.
 */
vup_status vup_propagate_weights(vup_grid g, int64_t K, const float *W, double *moments_raw,
                                 float *hist, vup_stream_t stream);

/*
 * vup_propagate_weights without any device allocation.  The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc once they are
 * running -- hosts with a fixed device-memory budget, allocators that forbid
 * growth after start-up, or code embedded in a runtime that owns the device
 * heap.  Inputs and outputs are exactly those of vup_propagate_weights (the
 * caller still owns W and the outputs; the grid is created beforehand).
 * Scratch: one device array of VUP_STATIC_SCRATCH_BYTES compiled into the
 * library; every GPU that loads libvup holds it until the process exits.
 * Each call needs K * (32 + 4 * n_bins) bytes of it at least; larger requests
 * return VUP_ERR_INVALID_ARG before any work is queued.
 * The first call on a device resolves the array's device address (set-up)
 * and keeps it for the life of the process; make that first call before any
 * stream capture.  A device reset (cudaDeviceReset) invalidates that address,
 * as it invalidates every grid: the library is not usable across one.  All calls share the array
 * and it keeps the last call's contents (nothing in it needs clearing): two
 * calls whose work overlaps on the GPU race, so serialise them (one stream).
 */
#define VUP_STATIC_SCRATCH_BYTES (16u << 20)
vup_status vup_propagate_weights_noalloc(vup_grid g, int64_t K, const float *W, double *moments_raw,
                                         float *hist, vup_stream_t stream);

/*
 * IPSA sensitivities (Sec. 5.2): derivatives of the raw moments M_j with
 * respect to each density's mu and sigma on every axis, for ndim == 2 grids
 * (and ndim == 1).  Gaussian and truncated-normal axes are differentiated
 * with their truncation bounds held fixed; uniform axes return 0.
 * W is recomputed, never stored.
 *   grad_moments NULL : full Jacobian, dmu/dsigma are [K][ndim][J] float
 *   grad_moments [K][J] double (device): vector-Jacobian product,
 *                        dmu/dsigma are [K][ndim] float,
 *                        dmu[k][d] = sum_j grad[k][j] dM_j/dmu_{k,d}
 * precision: VUP_FP32 or VUP_BF16X3 (VUP_FP64 for ndim == 1; the TF32 kinds
 * return VUP_ERR_UNSUPPORTED).
 */
vup_status vup_ipsa_sensitivity(vup_grid g, const vup_densities *d, vup_precision precision,
                                const double *grad_moments, float *dmu, float *dsigma,
                                vup_stream_t stream);

/*
 * Forward pass and IPSA sensitivities in one call: the outputs of
 * vup_propagate (moments_raw, moments_central, hist; each may be NULL) and of
 * vup_ipsa_sensitivity (grad_moments, dmu, dsigma as there) for the same
 * densities.  On a 2-D grid with VUP_FP32 or VUP_BF16X3 the densities are
 * prepared once and the moments are read off the sensitivity contraction of
 * the forward orientation (its first output plane is the moment contraction
 * itself), so no separate moment contraction runs; the results equal the two
 * separate calls'.  Other grids and precisions run the two calls in turn.
 * Errors as the two calls.
 */
vup_status vup_propagate_ipsa(vup_grid g, const vup_densities *d, vup_precision precision,
                              double *moments_raw, double *moments_central, float *hist,
                              const double *grad_moments, float *dmu, float *dsigma, vup_stream_t stream);

/*
 * Batched uneven propagation: n_inst independent instances (grid g[i] with
 * densities d[i]), the many-small-problems form of the Sec. 4 pipeline.  Every
 * stage runs as one launch over the work items of all instances, longest
 * items first (density preparation, the moment contraction, the FP64 finish,
 * the segmented histogram and its finish).
 *   g, d, moments_raw, hist : host arrays of length n_inst; moments_raw[i]
 *       ([K_i][J_i] double) and hist[i] ([K_i][B_i] float) are device
 *       pointers or NULL, laid out as in vup_propagate; moments_raw or hist
 *       may itself be NULL (no instance wants that output).
 *   precision : VUP_FP32 or VUP_BF16X3 (VUP_FP64 and the TF32 kinds:
 *       VUP_ERR_UNSUPPORTED).
 * Every grid must be 2-D with a model (VUP_ERR_STATE otherwise) and each
 * gathered-axis part of its histogram layout must fit one shared-memory tile
 * (704 rows; VUP_ERR_UNSUPPORTED otherwise).
 * The first call for a batch (same grids, densities, output pointers and
 * sizes) builds the work lists, chooses the contraction tile width for the
 * batch's shape (VUP_BF16X3: times tile-width caps 256, 128 and 64 once per
 * shape, replaying the whole batch; the choice is remembered for the process
 * and appended to the file named by the environment variable VUP_TUNE_CACHE,
 * if set, as one JSON object per line) and captures the launches into a CUDA
 * graph; later calls replay that graph on `stream`.  The first call is
 * synchronous and allocates; later calls allocate nothing and may be captured
 * into a caller's graph (their stage kernels are then captured directly; a
 * first call made while `stream` is capturing returns VUP_ERR_STATE).  Up to 8 batches are remembered.  Device conditions are
 * recorded per grid (VUP_ERR_EMPTY_SUPPORT) and, for an expired wait in the
 * contraction, in g[0]; read them with vup_sync.
 */
vup_status vup_propagate_batched(int n_inst, const vup_grid *g, const vup_densities *d,
                                 vup_precision precision, double *const *moments_raw,
                                 float *const *hist, vup_stream_t stream);

/*
 * ---- Coarse-grained IPSA quantities (Sec. 5.2) ----------------------------
 * The estimated value of column l is the model at the centre of its input
 * density, y(l) = M(l, 0) (the mean of every axis' density); the IPSA
 * probability matrix (Eq. IPSA) holds the probabilities of the deviations
 * dy = y - y(l); Eq. IPSAvar's local expected square deviation is
 * Delta^2 = E[dy^2] / 2.
 */

/*
 * The grid's built-in model at K arbitrary points: y[k] = M(x[k]; theta).
 *   x [K][ndim] double (device), y [K] double (device).
 * VUP_ERR_STATE if the grid has no built-in model (no vup_eval_model yet,
 * or outputs supplied with vup_set_outputs: evaluate y(l) yourself then).
 */
vup_status vup_model_at(vup_grid g, int64_t K, const double *x, double *y, vup_stream_t stream);

/*
 * Deviation moments about the estimated values:
 *   out[k][j-1] = sum_i W[k,i] (y_i - y_ref[k])^j,  j = 1..J (J of the grid),
 * formed from the raw moments of vup_propagate by the binomial expansion in
 * FP64.  Delta^2 = out[k][1] / 2.  moments_raw [K][J], y_ref [K], out [K][J],
 * all double (device).
 */
vup_status vup_deviation_moments(vup_grid g, int64_t K, const double *moments_raw, const double *y_ref,
                                 double *out, vup_stream_t stream);

/*
 * IPSA probability matrix (Eq. IPSA): every column of the output probability
 * matrix hist [K][B] (float, device, as written by vup_propagate on this
 * grid) translated by -y_ref[k] onto n_dbins deviation bins of width
 * (dhi - dlo) / n_dbins from dlo.  Output bin b stands for its centre
 * c_b = ymin + (b + 1/2)(ymax - ymin)/B; its mass goes to deviation bin
 * floor((c_b - y_ref[k] - dlo) / wd), clamped to [0, n_dbins - 1] so that
 * every column keeps its mass.  All decisions in FP64 with correctly rounded
 * operations; sums in increasing b.  out [K][n_dbins] float (device).
 * 1 <= n_dbins <= VUP_MAX_BINS, dlo < dhi finite.
 */
vup_status vup_ipsa_matrix(vup_grid g, int64_t K, const float *hist, const double *y_ref, int n_dbins, double dlo,
                           double dhi, float *out, vup_stream_t stream);

/*
 * Coarse-grained fields of K probability vectors hist [K][n_bins] (float,
 * device; an output histogram or an IPSA matrix), Sec. 5.2:
 *   argmax[k] (int32, or NULL): the first bin of maximum probability;
 *   ci[k][2] (int32, or NULL): the confidence-interval bins at `level`
 *       (0 < level < 1): the first bin whose cumulative mass exceeds
 *       (1 - level)/2 of the row total and the first whose cumulative mass
 *       reaches (1 + level)/2 of it (FP32 sums in bin order, each
 *       operation correctly rounded);
 *   global[n_bins] (double, or NULL): sum_k rho_k hist[k][b] / sum_k rho_k,
 *       the vector marginalised over l (FP64, summed in blocks of 64 rows);
 *       rho [K] double (device) or NULL for uniform weights.  The first call
 *       with a larger K x n_bins than before allocates library scratch.
 * At least one output must be requested.
 */
vup_status vup_sa_fields(int64_t K, int n_bins, const float *hist, double level, const double *rho,
                         int32_t *argmax, int32_t *ci, double *global, vup_stream_t stream);

/*
 * Bayes-inverted model matrix applied to the inputs (Sec. 3: the inverted
 * model matrix maps an output bin back to the input points that reach it,
 * each with posterior probability W[k,i] / H[k,b] by Bayes' theorem): the
 * posterior mean of every input axis per output bin,
 *   post[k][b][d] = sum_{i in bin b} W[k,i] x_{d,i} / H[k,b]  (0 where H = 0),
 * from FP32 segmented sums: one histogram pass for H and one per axis with
 * that axis' factors weighted by its coordinates (W is never formed).
 *   hist [K][B] float (device, or NULL): receives H as well;
 *   post [K][B][ndim] float (device).
 * ndim >= 2 (VUP_ERR_UNSUPPORTED for 1-D grids).  The first call with a
 * larger K than before allocates library scratch.
 */
vup_status vup_posterior_means(vup_grid g, const vup_densities *d, float *hist, float *post, vup_stream_t stream);

/*
 * What the calling thread's most recent vup_propagate_batched did:
 *   bn_cap  : tile-width cap of the contraction (256 / 128 / 64; 0 for FP32)
 *   source  : 0 replayed a remembered graph, 1 built a graph with a remembered
 *             tile-width choice, 2 built one after timing the candidates,
 *             -1 no call yet
 *   tune_ms : device time spent timing candidates in that call (0 if none)
 */
vup_status vup_batched_report(int *bn_cap, int *source, double *tune_ms);

/*
 * Wait for the grid's queued work on `stream` and return (and clear) the
 * first condition recorded on the device: VUP_OK, VUP_ERR_EMPTY_SUPPORT or
 * VUP_ERR_TIMEOUT.
 */
vup_status vup_sync(vup_grid g, vup_stream_t stream);

/*
 * Self-test of the bounded device-side waits: launches one CTA that waits on
 * an mbarrier nothing arrives at, polling `polls` times about 1 us apart
 * (1 <= polls <= 2^20, else VUP_ERR_INVALID_ARG), then records the expiry in
 * the grid's device status word and exits.  The next vup_sync(g) returns
 * VUP_ERR_TIMEOUT; the context stays usable.  This is the path every wait of
 * the contraction and histogram kernels takes on expiry.
 */
vup_status vup_selftest_wait(vup_grid g, uint32_t polls, vup_stream_t stream);

/* Grid facts after vup_eval_model / vup_set_outputs (host copies). */
typedef struct {
    int32_t ndim;
    int64_t n[3];
    int64_t N;
    int32_t n_bins;
    int32_t n_moments;
    double ymin, ymax, yscale;
    int32_t have_model;
    /* histogram walk chosen for the current model (2-D / 3-D grids):
     * layout 0 gathers the last axis, layout 1 axis 0 (2-D only); stream 0
     * walks sorted points, stream 1 sorted intervals (stretches of one bin
     * along the gathered axis, summed as differences of prefix sums), stream
     * 2 records (stretches of one line over a group of 4 consecutive bins,
     * monotone, five prefix sums for four bins).  Counts are those of the
     * chosen layout; hist_runs is 0 when the point and interval streams were
     * not built (the record stream was cheaper than both). */
    int32_t hist_layout, hist_stream;
    int64_t hist_runs, hist_intervals, hist_records;
    /* the power tables hold z = (y - yshift) / yscale: yshift is the point of
     * [ymin, ymax] nearest 0 (0 when the range holds 0), yscale = max |y - yshift| */
    double yshift;
} vup_grid_info_t;
vup_status vup_grid_info(vup_grid g, vup_grid_info_t *info);

/*
 * Histogram stream choice of a 2-D / 3-D grid: -1 (default) picks, per model,
 * the stream with the least estimated work; 0 forces the point stream, 1 the
 * interval stream, 2 the record stream.  All give H[k, b] of Eq. 4 (sums of
 * the same terms in a different order; the interval and record streams sum
 * stretches as differences of prefix sums, whose error is absolute, about
 * 2^-24 of a part's mass per stretch).  Takes effect for the current
 * model (queued on `stream`) and for later ones.  VUP_ERR_INVALID_ARG for
 * another value or a 1-D grid.
 */
vup_status vup_set_hist_stream(vup_grid g, int32_t stream_kind, vup_stream_t stream);

/* Form of vup_propagate_weights (_noalloc has its own): -1 (default) lets
 * the library choose; 0 the bin-sorted block walk (B <= 1024, N a multiple
 * of 4, W 16-byte aligned, ceil(K / 32) <= 65535); 1 a row of W per lane with shared-memory histogram rows
 * (B <= 1024); 2 the general form (any B).  A forced form that does not
 * apply to a call's B or K gives way to the next that does.  All give the
 * moments and H[k, b] of Eq. 4 from the same FP32 products (summed in a
 * different order).  VUP_ERR_INVALID_ARG for another value. */
vup_status vup_set_weights_form(vup_grid g, int32_t form);

/* Copy one of the grid's arrays into a caller device buffer (for checks).
 * which: 0 = y (double[N]), 1 = bin ids (int32[N]), 2 = sorted order
 * (int32[N], flat index of the t-th point in bin order), 3 = bin offsets
 * (int32[B+1]).  nbytes must equal the array's size. */
vup_status vup_grid_copy(vup_grid g, int which, void *dst_dev, size_t nbytes,
                         vup_stream_t stream);

/*
 * Per-kernel timing for measurement: while enabled, every kernel the library
 * launches is bracketed by CUDA events recorded on its launching stream.
 * vup_profile(1) clears the record and enables it, vup_profile(0) disables it.
 * vup_profile_read synchronises the device and writes a NUL-terminated JSON
 * object {"kernel": [launches, total_ms], ...} into buf (cap bytes).
 */
vup_status vup_profile(int enable);
vup_status vup_profile_read(char *buf, size_t cap);

/* The same record as a timeline: synchronises the device and writes a
 * NUL-terminated JSON array [[name, stream, launches, begin_ms, end_ms], ...]
 * in launch order into buf (cap bytes); times are relative to the first
 * record's begin event, stream numbers count the distinct launching streams
 * in order of first use.  VUP_ERR_INVALID_ARG if buf is null or too small. */
vup_status vup_profile_timeline(char *buf, size_t cap);

/*
 * Measured ceiling of a CUDA-core resource, the denominator of the roofline
 * fractions of kernels bound by it (not part of the method):
 *   kind 0: FP32 fused multiply-add throughput, FLOP/s (an FMA counts two);
 *   kind 1: shared-memory gathers of 512-byte rows by whole warps (16 bytes
 *           per lane, a data-dependent row per warp), bytes/s through the
 *           SM's L1 data pipe.
 * Runs a few milliseconds of work on every SM of the current device on
 * `stream`, waits for it and writes the rate to *value (host).  Allocates
 * and frees a small device buffer.
 */
vup_status vup_measure_peak(int kind, vup_stream_t stream, double *value);

/* Static description of a status code. */
const char *vup_status_string(vup_status s);

/*
 * The calling thread's last CUDA failure as text ("error name: failing call
 * (file:line)"), set whenever a call returns VUP_ERR_CUDA or VUP_ERR_OOM; a
 * thread-local static buffer owned by the library, valid until the thread's
 * next failing call.  Empty if no call of this thread has failed.
 */
const char *vup_last_error_detail(void);

/*
 * Allocation-failure hook for tests of the out-of-memory paths (not part of
 * the method): after `after` more device allocations by the library succeed,
 * every later one fails as if the device were out of memory, until the hook
 * is disarmed with after < 0 (its state at load).  Process-wide.  A call
 * whose allocation fails returns VUP_ERR_OOM before it queues any work that
 * writes the caller's outputs, and the grid stays usable.
 */
vup_status vup_debug_fail_alloc(int64_t after);

/* Library version string. */
const char *vup_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VUP_H */
