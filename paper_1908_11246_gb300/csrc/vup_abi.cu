// C ABI of libvup: argument checking, grid lifetime, scratch management and
// the order in which the hot-path kernels are queued.
#include "vup_internal.cuh"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

static thread_local char g_last_err[512];

void vup_set_last_cuda_error(cudaError_t e, const char *expr, const char *file, int line) {
    snprintf(g_last_err, sizeof(g_last_err), "%s: %s (%s:%d)", cudaGetErrorName(e), expr, file, line);
}

// Allocation-failure hook: < 0 disarmed; otherwise the number of device
// allocations that still succeed before every later one fails.
static std::atomic<int64_t> g_fail_after{-1};

cudaError_t vup_dev_malloc_raw(void **p, size_t bytes) {
    int64_t n = g_fail_after.load();
    while (n >= 0) {
        if (n == 0) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_fail_after.compare_exchange_weak(n, n - 1)) break;
    }
    return cudaMalloc(p, bytes);
}

extern "C" vup_status vup_debug_fail_alloc(int64_t after) {
    g_fail_after.store(after < 0 ? -1 : after);
    return VUP_OK;
}

vup_status devbuf_reserve(DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return VUP_OK;
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    void *p = nullptr;
    cudaError_t e = vup_dev_malloc(&p, bytes < 256 ? 256 : bytes);
    if (e != cudaSuccess) {
        vup_set_last_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        cudaGetLastError();
        return VUP_ERR_OOM;
    }
    b.p = p;
    b.bytes = bytes;
    return VUP_OK;
}

void devbuf_free(DevBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// ---- per-kernel timing registry -------------------------------------------
namespace {
struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
    int launches;
    cudaStream_t stream;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_prof_pool;

cudaEvent_t prof_event() {
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

ProfScope::ProfScope(const char *n, cudaStream_t s, int l) : name(n), stream(s), launches(l), slot(-1) {
    if (!g_prof_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfRec r{n, prof_event(), prof_event(), l, s};
    cudaEventRecord(r.a, s);
    g_prof_recs.push_back(r);
    slot = (int)g_prof_recs.size() - 1;
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (slot < (int)g_prof_recs.size()) {
        g_prof_recs[slot].launches = launches;  // a scope may count its launches as it goes
        cudaEventRecord(g_prof_recs[slot].b, stream);
    }
}

bool vup_profiling() { return g_prof_on; }

extern "C" vup_status vup_profile(int enable) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (enable) {
        for (auto &r : g_prof_recs) {
            g_prof_pool.push_back(r.a);
            g_prof_pool.push_back(r.b);
        }
        g_prof_recs.clear();
    }
    g_prof_on = enable != 0;
    return VUP_OK;
}

extern "C" vup_status vup_profile_read(char *buf, size_t cap) {
    if (!buf || cap < 3) return VUP_ERR_INVALID_ARG;
    VUP_CHECK_CUDA(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::map<std::string, std::pair<long, double>> agg;
    for (auto &r : g_prof_recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        auto &e = agg[r.name];
        e.first += r.launches;
        e.second += ms;
    }
    std::string out = "{";
    bool first = true;
    for (auto &kv : agg) {
        char tmp[256];
        snprintf(tmp, sizeof(tmp), "%s\"%s\": [%ld, %.6f]", first ? "" : ", ", kv.first.c_str(), kv.second.first,
                 kv.second.second);
        out += tmp;
        first = false;
    }
    out += "}";
    if (out.size() + 1 > cap) return VUP_ERR_INVALID_ARG;
    memcpy(buf, out.c_str(), out.size() + 1);
    return VUP_OK;
}

extern "C" vup_status vup_profile_timeline(char *buf, size_t cap) {
    if (!buf || cap < 3) return VUP_ERR_INVALID_ARG;
    VUP_CHECK_CUDA(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::vector<cudaStream_t> streams;
    std::string out = "[";
    bool first = true;
    for (auto &r : g_prof_recs) {
        float t0 = 0.f, t1 = 0.f;
        if (cudaEventElapsedTime(&t0, g_prof_recs[0].a, r.a) != cudaSuccess ||
            cudaEventElapsedTime(&t1, g_prof_recs[0].a, r.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        size_t si = 0;
        while (si < streams.size() && streams[si] != r.stream) ++si;
        if (si == streams.size()) streams.push_back(r.stream);
        char tmp[256];
        snprintf(tmp, sizeof(tmp), "%s[\"%s\", %zu, %d, %.6f, %.6f]", first ? "" : ", ", r.name, si, r.launches, t0,
                 t1);
        out += tmp;
        first = false;
    }
    out += "]";
    if (out.size() + 1 > cap) return VUP_ERR_INVALID_ARG;
    memcpy(buf, out.c_str(), out.size() + 1);
    return VUP_OK;
}

int vup_num_sms() {
    int dev = 0, n = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

int vup_hist_chunks_for(int64_t N, int P);
int vup_hist_parts_for(int64_t n_last, int n_bins);
int vup_hist_rec_chunks_for(int n_chunks);

extern "C" const char *vup_status_string(vup_status s) {
    switch (s) {
    case VUP_OK: return "VUP_OK";
    case VUP_ERR_INVALID_ARG: return "VUP_ERR_INVALID_ARG: invalid argument";
    case VUP_ERR_CUDA: return "VUP_ERR_CUDA: a CUDA call failed";
    case VUP_ERR_OOM: return "VUP_ERR_OOM: device allocation failed";
    case VUP_ERR_STATE: return "VUP_ERR_STATE: grid has no model outputs (call vup_eval_model)";
    case VUP_ERR_EMPTY_SUPPORT: return "VUP_ERR_EMPTY_SUPPORT: a density holds no grid point";
    case VUP_ERR_TIMEOUT: return "VUP_ERR_TIMEOUT: a bounded device wait expired";
    case VUP_ERR_BOUNDS: return "VUP_ERR_BOUNDS: a device bounds check of the debug build failed";
    case VUP_ERR_UNSUPPORTED: return "VUP_ERR_UNSUPPORTED: not implemented for these arguments";
    }
    return "unknown vup_status";
}

extern "C" const char *vup_version(void) { return "vup-gb300 0.1 (sm_103a)"; }

extern "C" const char *vup_last_error_detail(void) { return g_last_err; }

static void free_grid(vup_grid g) {
    cudaFree(g->y);
    cudaFree(g->axis_terms);
    cudaFree(g->ext);
    cudaFree(g->bins);
    cudaFree(g->perm);
    cudaFree(g->offsets);
    {  // the built layout's arrays (hl[1] aliases them)
        auto &L = g->hl[0];
        if (L.perm != g->perm) cudaFree(L.perm);
        cudaFree(L.keys_own);
        cudaFree(L.koff);
        cudaFree(L.key_chunks);
        cudaFree(L.hpt);
        cudaFree(L.run_start);
        cudaFree(L.run_rest);
        cudaFree(L.run_bin);
        cudaFree(L.n_runs);
        cudaFree(L.chunk_pt);
        cudaFree(L.chunk_run);
        cudaFree(L.chunk_bin);
        cudaFree(L.ipt);
        cudaFree(L.iv_rest);
        cudaFree(L.n_iv);
        cudaFree(L.chunk_iv);
        cudaFree(L.n_rec);
        cudaFree(L.rec_chunk);
        cudaFree(L.rec_chunk_grp);
        devbuf_free(L.rec);
        devbuf_free(L.rec_rest);
        devbuf_free(L.rec_goff);
        devbuf_free(L.rec_gch);
    }
    cudaFree(g->hist_sel);
    if (g->side) cudaStreamDestroy(g->side);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    if (g->ev_rec) cudaEventDestroy(g->ev_rec);
    if (g->ev_lay) cudaEventDestroy(g->ev_lay);
    if (g->ev_dens) cudaEventDestroy(g->ev_dens);
    if (g->ev_pre) cudaEventDestroy(g->ev_pre);
    if (g->ev_mom) cudaEventDestroy(g->ev_mom);
    if (g->ev_mfin) cudaEventDestroy(g->ev_mfin);
    if (g->side2) cudaStreamDestroy(g->side2);
    cudaFree(g->ydev_scale);
    cudaFree(g->dstatus);
    for (int o = 0; o < kNumOrient; ++o) {
        cudaFree(g->ztf_hi[o]);
        cudaFree(g->ztf_lo[o]);
        cudaFree(g->zs[o]);
        cudaFree(g->zt_hi[o]);
        cudaFree(g->zt_lo[o]);
    }
    devbuf_free(g->sort_counts);
    devbuf_free(g->scan_tmp);
    devbuf_free(g->lay_tmp);
    devbuf_free(g->rec_tmp);
    devbuf_free(g->dconst);
    devbuf_free(g->dstats);
    devbuf_free(g->dpart);
    devbuf_free(g->ftab);
    devbuf_free(g->atab_hi);
    devbuf_free(g->atab_lo);
    devbuf_free(g->partials);
    devbuf_free(g->hist_part);
    devbuf_free(g->hist_direct);
    devbuf_free(g->hist_prefix);
    devbuf_free(g->ipsa_part);
    devbuf_free(g->atf_hi);
    devbuf_free(g->atf_lo);
    devbuf_free(g->wsort_pt);
    devbuf_free(g->wsort_z);
    devbuf_free(g->wsort_fix);
    delete g;
}

extern "C" vup_status vup_grid_create(int ndim, const int64_t *n, const double *lo, const double *hi,
                                      vup_grid *out) {
    if (!out || !n || !lo || !hi || ndim < 1 || ndim > 3) return VUP_ERR_INVALID_ARG;
    *out = nullptr;
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) {
        if (n[d] < 1 || n[d] > VUP_MAX_AXIS_POINTS) return VUP_ERR_INVALID_ARG;
        if (!isfinite(lo[d]) || !isfinite(hi[d]) || !(lo[d] < hi[d])) return VUP_ERR_INVALID_ARG;
        N *= n[d];
    }
    if (N >= ((int64_t)1 << 31) - 1) return VUP_ERR_INVALID_ARG;
    vup_grid g = new vup_grid_s();
    cudaGetDevice(&g->device);
    g->ndim = ndim;
    g->N = N;
    for (int d = 0; d < ndim; ++d) {
        g->n[d] = n[d];
        g->lo[d] = lo[d];
        g->hi[d] = hi[d];
    }
    // orientation 0: reduce over the last axis; orientation 1: over axis 0 (2-D)
    for (int o = 0; o < 2; ++o) {
        Orient &ori = g->orient[o];
        ori.red_axis0 = o == 0 ? ndim - 1 : 0;
        ori.R = g->n[ori.red_axis0];
        ori.R_pad = ceil_div64(ori.R, 64) * 64;
        ori.Q = N / ori.R;
        ori.NC = ori.Q * 4;
        ori.n_rest_axes = 0;
        ori.rest_axes[0] = ori.rest_axes[1] = -1;
        ori.rest_n[0] = ori.rest_n[1] = 1;
        for (int d = 0; d < ndim; ++d)
            if (d != ori.red_axis0 && ori.n_rest_axes < 2) {
                ori.rest_n[ori.n_rest_axes] = g->n[d];
                ori.rest_axes[ori.n_rest_axes++] = d;
            }
    }
    int p_all = 1;  // the most parts any layout of this grid can have
    for (int l = 0; l < (ndim == 2 ? 2 : 1); ++l)
        p_all = std::max(p_all, vup_hist_parts_for(g->n[l == 0 ? ndim - 1 : 0], 1));
    g->n_chunks = vup_hist_chunks_for(N, p_all);
    g->n_chunks_rec = vup_hist_rec_chunks_for(g->n_chunks);
    const int C = g->n_chunks;
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes) \
    if (e == cudaSuccess) e = vup_dev_malloc((void **)&(ptr), (bytes))
    ALLOC(g->y, sizeof(double) * N);
    ALLOC(g->axis_terms, sizeof(double2) * (size_t)(g->n[0] + (ndim > 1 ? g->n[1] : 0) + (ndim > 2 ? g->n[2] : 0)));
    ALLOC(g->ext, sizeof(unsigned long long) * 3);  // range keys (min, max) and a grid-barrier counter
    ALLOC(g->bins, sizeof(int32_t) * N);
    ALLOC(g->perm, sizeof(int32_t) * N);
    g->n_layouts = ndim == 2 ? 2 : 1;
    int p_max = 1;
    for (int l = 0; l < g->n_layouts; ++l) {
        auto &L = g->hl[l];
        L.last_axis = l == 0 ? ndim - 1 : 0;
        L.n_last = g->n[L.last_axis];
        p_max = std::max(p_max, vup_hist_parts_for(L.n_last, 1));
    }
    {
        auto &L = g->hl[0];  // arrays of the one layout built per model
        ALLOC(L.hpt, sizeof(uint32_t) * (N + 512));  // tail slack for whole staged windows
        ALLOC(L.run_start, sizeof(int32_t) * (N + 1));
        ALLOC(L.run_rest, sizeof(int32_t) * N);
        ALLOC(L.run_bin, sizeof(int32_t) * N);
        ALLOC(L.n_runs, sizeof(int32_t));
        ALLOC(L.chunk_pt, sizeof(int32_t) * (p_max * C + 1));
        ALLOC(L.chunk_run, sizeof(int32_t) * (p_max * C + 1));
        ALLOC(L.chunk_bin, sizeof(int32_t) * 2 * p_max * C);
        if (ndim >= 2) {
            ALLOC(L.perm, sizeof(int32_t) * N);
            ALLOC(L.keys_own, sizeof(int32_t) * N);
            ALLOC(L.ipt, sizeof(uint2) * (N + 128));  // tail slack for whole staged windows
            ALLOC(L.iv_rest, sizeof(int32_t) * N);
            ALLOC(L.n_iv, sizeof(int32_t));
            ALLOC(L.chunk_iv, sizeof(int32_t) * (p_max * C + 1));
            ALLOC(L.n_rec, sizeof(int32_t));
            ALLOC(L.rec_chunk, sizeof(int32_t) * (p_max * g->n_chunks_rec + 1));
            ALLOC(L.rec_chunk_grp, sizeof(int32_t) * 2 * p_max * g->n_chunks_rec);
            // words past the stream's end are read by whole-window staging and
            // masked; zero keeps their rest codes valid indices
            if (e == cudaSuccess) e = cudaMemset(L.ipt, 0, sizeof(uint2) * (N + 128));
        } else {
            L.perm = g->perm;
        }
    }
    if (g->n_layouts > 1) {
        auto &A = g->hl[0];
        auto &L = g->hl[1];
        L.perm = A.perm;
        L.keys_own = A.keys_own;
        L.hpt = A.hpt;
        L.run_start = A.run_start;
        L.run_rest = A.run_rest;
        L.run_bin = A.run_bin;
        L.n_runs = A.n_runs;
        L.chunk_pt = A.chunk_pt;
        L.chunk_run = A.chunk_run;
        L.chunk_bin = A.chunk_bin;
        L.ipt = A.ipt;
        L.iv_rest = A.iv_rest;
        L.n_iv = A.n_iv;
        L.chunk_iv = A.chunk_iv;
        L.n_rec = A.n_rec;
        L.rec_chunk = A.rec_chunk;
        L.rec_chunk_grp = A.rec_chunk_grp;
    }
    ALLOC(g->hist_sel, sizeof(int32_t) * 8);
    ALLOC(g->ydev_scale, sizeof(double) * kScaleSlots);
    ALLOC(g->dstatus, sizeof(int));
#undef ALLOC
    if (e == cudaSuccess) e = cudaMemset(g->dstatus, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(g->hist_sel, 0, sizeof(int32_t) * 8);
    if (e != cudaSuccess) {
        vup_set_last_cuda_error(e, "vup_grid_create", __FILE__, __LINE__);
        cudaGetLastError();
        free_grid(g);
        return e == cudaErrorMemoryAllocation ? VUP_ERR_OOM : VUP_ERR_CUDA;
    }
    *out = g;
    return VUP_OK;
}

extern "C" vup_status vup_grid_destroy(vup_grid g) {
    if (!g) return VUP_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    free_grid(g);
    return VUP_OK;
}

static vup_status model_ready(vup_grid g, int n_bins, int n_moments) {
    if (n_bins < 1 || n_bins > VUP_MAX_BINS || n_moments < 1 || n_moments > VUP_MAX_MOMENTS)
        return VUP_ERR_INVALID_ARG;
    if (g->B_cap < n_bins) {
        cudaFree(g->offsets);
        g->offsets = nullptr;
        VUP_CHECK_CUDA(vup_dev_malloc(&g->offsets, sizeof(int32_t) * (n_bins + 1)));
        g->B_cap = n_bins;
    }
    g->B = n_bins;
    g->J = n_moments;
    return VUP_OK;
}

static vup_status finish_model(vup_grid g, cudaStream_t s) {
    vup_status st = vup_launch_grid_finish(g, s);
    if (st != VUP_OK) return st;
    // power tables are built on first use by the contraction that needs them
    g->have_model = 1;
    ++g->model_gen;
    return VUP_OK;
}

static bool model_ndim_ok(int model_id, int ndim) {
    switch (model_id) {
    case VUP_MODEL_SIN_QUAD_1D: return ndim == 1;
    case VUP_MODEL_SIN_SIN2_2D:
    case VUP_MODEL_OSCILLATOR_2D:
    case VUP_MODEL_IPSA_EXAMPLE_2D: return ndim == 2;
    case VUP_MODEL_MIXED_3D: return ndim == 3;
    case VUP_MODEL_POLY: return ndim >= 1 && ndim <= 3;
    default: return false;
    }
}

extern "C" vup_status vup_eval_model(vup_grid g, int model_id, const double *theta, int n_theta, int n_bins,
                                     int n_moments, vup_stream_t stream) {
    if (!g || n_theta < 0 || n_theta > 8 || (n_theta > 0 && !theta)) return VUP_ERR_INVALID_ARG;
    if (!model_ndim_ok(model_id, g->ndim)) return VUP_ERR_INVALID_ARG;
    double th[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < n_theta; ++q) {
        if (!isfinite(theta[q])) return VUP_ERR_INVALID_ARG;
        th[q] = theta[q];
    }
    vup_status st = model_ready(g, n_bins, n_moments);
    if (st != VUP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    g->have_model = 0;
    g->model_id = model_id;
    for (int q = 0; q < 8; ++q) g->theta[q] = th[q];
    st = vup_launch_model_eval(g, model_id, th, s);
    if (st != VUP_OK) return st;
    return finish_model(g, s);
}

extern "C" vup_status vup_set_outputs(vup_grid g, const double *y_dev, int n_bins, int n_moments,
                                      vup_stream_t stream) {
    if (!g || !y_dev) return VUP_ERR_INVALID_ARG;
    vup_status st = model_ready(g, n_bins, n_moments);
    if (st != VUP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    g->have_model = 0;
    g->model_id = 0;
    VUP_CHECK_CUDA(cudaMemcpyAsync(g->y, y_dev, sizeof(double) * g->N, cudaMemcpyDeviceToDevice, s));
    g->range_ready = 0;
    return finish_model(g, s);
}

vup_status vup_check_dens(vup_grid g, const vup_densities *d) {
    if (!d || d->K < 1 || d->K > VUP_MAX_DENSITIES || d->ndim != g->ndim) return VUP_ERR_INVALID_ARG;
    if (!d->kind || !d->mu || !d->sigma) return VUP_ERR_INVALID_ARG;
    if ((d->lo == nullptr) != (d->hi == nullptr)) return VUP_ERR_INVALID_ARG;
    return VUP_OK;
}

// Per-K scratch: density constants, factor tables, split A tables, partials.
vup_status vup_reserve_k(vup_grid g, int64_t K, bool bf16, bool ipsa, bool tf32) {
    const int64_t K_pad = ceil_div64(K, 128) * 128;
    const int nd = g->ndim;
    vup_status st;
    if ((st = devbuf_reserve(g->dconst, sizeof(DensConst) * K_pad * nd)) != VUP_OK) return st;
    if ((st = devbuf_reserve(g->dstats, sizeof(DensStats) * K_pad * nd)) != VUP_OK) return st;
    if ((st = devbuf_reserve(g->ftab, sizeof(float) * K_pad * vup_ftab_floats(g))) != VUP_OK) return st;
    if (nd >= 2) {
        const int64_t nct = std::max(vup_simt_col_tiles(g->orient[0]), vup_tc_col_tiles_max(g->orient[vup_tc_orient(g)]));
        if ((st = devbuf_reserve(g->partials, sizeof(float) * 4 * K_pad * nct)) != VUP_OK) return st;
        // partial rows of cut keys (2 per chunk) or cut record groups (2 x 8 bins per record chunk)
        const size_t part_rows = std::max<size_t>(2 * (size_t)g->n_chunks, 16 * (size_t)g->n_chunks_rec);
        if ((st = devbuf_reserve(g->hist_part, sizeof(float) * part_rows * K_pad * g->hist_P)) != VUP_OK)
            return st;
        if ((st = devbuf_reserve(g->hist_direct, sizeof(float) * (size_t)g->hist_P * g->B * K_pad)) != VUP_OK)
            return st;
        {
            int64_t rows = 1;
            for (int l = 0; l < g->n_layouts; ++l) rows = std::max(rows, g->hl[l].part_rows);
            if ((st = devbuf_reserve(g->hist_prefix, sizeof(float) * (size_t)g->hist_P * K_pad * (rows + 1))) != VUP_OK)
                return st;
        }
        if (tf32) {
            const size_t a = (size_t)K_pad * g->orient[vup_tc_orient(g)].R_pad;
            if ((st = devbuf_reserve(g->atf_hi, sizeof(float) * a)) != VUP_OK) return st;
            if ((st = devbuf_reserve(g->atf_lo, sizeof(float) * a)) != VUP_OK) return st;
        }
        if (bf16) {
            size_t a = (size_t)K_pad * g->orient[vup_tc_orient(g)].R_pad +
                       (ipsa ? (size_t)K_pad * g->orient[1].R_pad : 0);
            if ((st = devbuf_reserve(g->atab_hi, sizeof(__nv_bfloat16) * a)) != VUP_OK) return st;
            if ((st = devbuf_reserve(g->atab_lo, sizeof(__nv_bfloat16) * a)) != VUP_OK) return st;
        }
        if (ipsa) {
            int64_t n0 = std::max(vup_simt_col_tiles(g->orient[0]), vup_tc_col_tiles_max(g->orient[0]));
            int64_t n1 = std::max(vup_simt_col_tiles(g->orient[1]), vup_tc_col_tiles_max(g->orient[1]));
            if ((st = devbuf_reserve(g->ipsa_part, sizeof(float) * 4 * 3 * K_pad * (n0 + n1))) != VUP_OK)
                return st;
        }
    }
    g->K_cap = std::max(g->K_cap, K);
    return VUP_OK;
}

// Sensitivity outputs of a fused forward + IPSA call (vup_propagate_ipsa).
struct IpsaOut {
    const double *grad;
    float *dmu, *dsg;
};

// The forward pass of a 2-D / 3-D grid; with `ip` (2-D, FP32 or BF16x3) also
// the IPSA sensitivities, from one density preparation, the moments read off
// the first output plane of the forward orientation's sensitivity contraction.
static vup_status propagate_nd(vup_grid g, const vup_densities *d, vup_precision precision, double *moments_raw,
                               double *moments_central, float *hist, cudaStream_t s, const IpsaOut *ip) {
    vup_status st;
    const int64_t K = d->K;
    const bool bf16 = precision == VUP_BF16X3;
    const bool tf32 = precision == VUP_TF32 || precision == VUP_TF32X3;
    const bool want_m = moments_raw || moments_central;
    const bool fuse = ip != nullptr;
    if ((st = vup_reserve_k(g, K, bf16, fuse, tf32)) != VUP_OK) return st;
    // the histogram layout (when not built for this model yet) on the second
    // stream, beside the density preparation and the contraction
    bool forked = false;
    if (hist && !g->layout_valid) {
        if (!g->side) {
            // high priority: the layout's small latency-bound launches take SMs as
            // they free up, ahead of the main stream's large kernels
            int lo_prio = 0, hi_prio = 0;
            VUP_CHECK_CUDA(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
            VUP_CHECK_CUDA(cudaStreamCreateWithPriority(&g->side, cudaStreamNonBlocking, hi_prio));
            VUP_CHECK_CUDA(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
            VUP_CHECK_CUDA(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
            VUP_CHECK_CUDA(cudaEventCreateWithFlags(&g->ev_rec, cudaEventDisableTiming));
            VUP_CHECK_CUDA(cudaEventCreateWithFlags(&g->ev_lay, cudaEventDisableTiming));
        }
        VUP_CHECK_CUDA(cudaEventRecord(g->ev_fork, s));
        forked = true;
    }
    // every return below joins the second stream back into the caller's
    struct Join {
        bool on;
        cudaStream_t s;
        cudaEvent_t e;
        ~Join() {
            if (on) cudaStreamWaitEvent(s, e, 0);
        }
    } join{forked, s, g->ev_join}, join_fin{false, s, g->ev_mfin};
    const int to = vup_tc_orient(g);
    if (fuse) {
        // both orientations' tables and split factors, and the statistics the
        // sensitivities need
        for (int o = 0; o < 2; ++o)
            if ((st = vup_build_tables(g, o, bf16 ? 1 : 0, s)) != VUP_OK) return st;
        if ((st = vup_density_prep(g, d, bf16 ? 3 : 0, s, false, true)) != VUP_OK) return st;
    } else {
        if (want_m && (st = vup_build_tables(g, (bf16 || tf32) ? to : kOrientLast, tf32 ? 2 : (bf16 ? 1 : 0), s)) !=
                          VUP_OK)
            return st;
        if ((st = vup_density_prep(g, d, ((bf16 || tf32) && want_m) ? (1 << to) : 0, s, tf32)) != VUP_OK) return st;
    }
    if (forked) {
        // the layout's launches are enqueued after the density preparation's, so
        // that the main stream's work is not held behind their host-side cost
        VUP_CHECK_CUDA(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
        vup_status lst = vup_build_layout(g, g->side, false, g->ev_rec, g->ev_lay);
        VUP_CHECK_CUDA(cudaEventRecord(g->ev_join, g->side));
        if (lst != VUP_OK) return lst;
    }
    // the histogram's prefix-sum tiles on a third stream, beside the
    // contraction (they need the densities and the layout choice only)
    bool prefix_ready = false;
    if (hist && forked && want_m) {
        if (!g->side2) {
            VUP_CHECK_CUDA(cudaStreamCreateWithFlags(&g->side2, cudaStreamNonBlocking));
            VUP_CHECK_CUDA(cudaEventCreateWithFlags(&g->ev_dens, cudaEventDisableTiming));
            VUP_CHECK_CUDA(cudaEventCreateWithFlags(&g->ev_pre, cudaEventDisableTiming));
            VUP_CHECK_CUDA(cudaEventCreateWithFlags(&g->ev_mom, cudaEventDisableTiming));
            VUP_CHECK_CUDA(cudaEventCreateWithFlags(&g->ev_mfin, cudaEventDisableTiming));
            join_fin.e = g->ev_mfin;
        }
        VUP_CHECK_CUDA(cudaEventRecord(g->ev_dens, s));
        VUP_CHECK_CUDA(cudaStreamWaitEvent(g->side2, g->ev_dens, 0));
        VUP_CHECK_CUDA(cudaStreamWaitEvent(g->side2, g->ev_lay, 0));
        prefix_ready = vup_hist_prefix(g, K, g->side2);
        VUP_CHECK_CUDA(cudaEventRecord(g->ev_pre, g->side2));
    }
    // fused: the sensitivity partials of both orientations ([3][tiles][K_pad][4]
    // each, orientation 1 after orientation 0), the forward orientation first
    const int fo = bf16 ? to : 0;
    float *ipart[2] = {nullptr, nullptr};
    int64_t inct[2] = {0, 0};
    if (fuse) {
        const int64_t K_pad = ceil_div64(K, 128) * 128;
        for (int o = 0; o < 2; ++o)
            inct[o] = bf16 ? vup_tc_col_tiles(g->orient[o], K) : vup_simt_col_tiles(g->orient[o]);
        ipart[0] = (float *)g->ipsa_part.p;
        ipart[1] = ipart[0] + (size_t)3 * inct[0] * K_pad * 4;
    }
    if (want_m || fuse) {
        int64_t nct;
        const float *mpart = nullptr;
        if (fuse) {
            // w, w u, w u^2 of the forward orientation: plane 0 is the moment contraction
            st = bf16 ? vup_moments_tc(g, K, fo, 3, ipart[fo], s) : vup_moments_simt(g, K, fo, 3, ipart[fo], s);
            if (st != VUP_OK) return st;
            nct = inct[fo];
            mpart = ipart[fo];
        } else if (bf16 || tf32) {
            if ((st = vup_moments_tc(g, K, to, 1, (float *)g->partials.p, s, tf32 ? 1 : 0,
                                     precision == VUP_TF32 ? 1 : 3)) != VUP_OK)
                return st;
            nct = vup_tc_col_tiles(g->orient[to], K);
        } else {
            if ((st = vup_moments_simt(g, K, 0, 1, (float *)g->partials.p, s)) != VUP_OK) return st;
            nct = vup_simt_col_tiles(g->orient[0]);
        }
        if (!want_m) {
        } else if (prefix_ready) {
            // the FP64 finish on the third stream: the histogram does not need it
            VUP_CHECK_CUDA(cudaEventRecord(g->ev_mom, s));
            VUP_CHECK_CUDA(cudaStreamWaitEvent(g->side2, g->ev_mom, 0));
            join_fin.on = true;
            st = vup_moments_finish(g, K, (int)nct, moments_raw, moments_central, g->side2, mpart);
            VUP_CHECK_CUDA(cudaEventRecord(g->ev_mfin, g->side2));
            if (st != VUP_OK) return st;
        } else if ((st = vup_moments_finish(g, K, (int)nct, moments_raw, moments_central, s, mpart)) != VUP_OK) {
            return st;
        }
    }
    if (hist) {
        // the record-stream histogram waits for the records only; the other
        // streams' kernels (and the finish) for the whole layout
        if (forked) VUP_CHECK_CUDA(cudaStreamWaitEvent(s, g->ev_rec, 0));
        if (prefix_ready) VUP_CHECK_CUDA(cudaStreamWaitEvent(s, g->ev_pre, 0));
        if ((st = vup_hist_fused(g, K, hist, s, nullptr, false, forked ? g->ev_join : nullptr, prefix_ready)) !=
            VUP_OK)
            return st;
        join.on = false;
    }
    if (fuse) {
        // the other orientation's sensitivity contraction, then the combine
        const int oo = 1 - fo;
        st = bf16 ? vup_moments_tc(g, K, oo, 3, ipart[oo], s) : vup_moments_simt(g, K, oo, 3, ipart[oo], s);
        if (st != VUP_OK) return st;
        if ((st = vup_ipsa_finish(g, K, (int)inct[0], (int)inct[1], ip->grad, ip->dmu, ip->dsg, s)) != VUP_OK)
            return st;
    }
    return VUP_OK;
}

extern "C" vup_status vup_propagate(vup_grid g, const vup_densities *d, vup_precision precision,
                                    double *moments_raw, double *moments_central, float *hist,
                                    vup_stream_t stream) {
    if (!g) return VUP_ERR_INVALID_ARG;
    vup_status st = vup_check_dens(g, d);
    if (st != VUP_OK) return st;
    if (precision < VUP_FP64 || precision > VUP_TF32X3) return VUP_ERR_INVALID_ARG;
    if (!g->have_model) return VUP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->ndim == 1) {
        if (precision != VUP_FP64 && precision != VUP_FP32) return VUP_ERR_UNSUPPORTED;
        return vup_propagate_1d(g, d, moments_raw, moments_central, hist, s);
    }
    if (precision == VUP_FP64) return VUP_ERR_UNSUPPORTED;
    return propagate_nd(g, d, precision, moments_raw, moments_central, hist, s, nullptr);
}

extern "C" vup_status vup_propagate_weights(vup_grid g, int64_t K, const float *W, double *moments_raw,
                                            float *hist, vup_stream_t stream) {
    if (!g || !W || K < 1 || K > VUP_MAX_DENSITIES) return VUP_ERR_INVALID_ARG;
    if (!g->have_model) return VUP_ERR_STATE;
    return vup_weights_path(g, K, W, moments_raw, hist, (cudaStream_t)stream);
}

extern "C" vup_status vup_ipsa_sensitivity(vup_grid g, const vup_densities *d, vup_precision precision,
                                           const double *grad_moments, float *dmu, float *dsigma,
                                           vup_stream_t stream) {
    if (!g || !dmu || !dsigma) return VUP_ERR_INVALID_ARG;
    vup_status st = vup_check_dens(g, d);
    if (st != VUP_OK) return st;
    if (precision < VUP_FP64 || precision > VUP_TF32X3) return VUP_ERR_INVALID_ARG;
    if (precision == VUP_TF32 || precision == VUP_TF32X3) return VUP_ERR_UNSUPPORTED;
    if (!g->have_model) return VUP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->ndim == 1) {
        if (precision == VUP_BF16X3) return VUP_ERR_UNSUPPORTED;
        return vup_ipsa_1d(g, d, grad_moments, dmu, dsigma, s);
    }
    if (g->ndim != 2 || precision == VUP_FP64) return VUP_ERR_UNSUPPORTED;
    const int64_t K = d->K;
    const bool bf16 = precision == VUP_BF16X3;
    if ((st = vup_reserve_k(g, K, bf16, true)) != VUP_OK) return st;
    if ((st = vup_build_tables(g, 0, bf16 ? 1 : 0, s)) != VUP_OK) return st;
    if ((st = vup_build_tables(g, 1, bf16 ? 1 : 0, s)) != VUP_OK) return st;
    if ((st = vup_density_prep(g, d, bf16 ? 3 : 0, s, false, true)) != VUP_OK) return st;
    const int64_t K_pad = ceil_div64(K, 128) * 128;
    float *p0 = (float *)g->ipsa_part.p;
    int64_t n0, n1;
    if (bf16) {
        n0 = vup_tc_col_tiles(g->orient[0], K);
        n1 = vup_tc_col_tiles(g->orient[1], K);
    } else {
        n0 = vup_simt_col_tiles(g->orient[0]);
        n1 = vup_simt_col_tiles(g->orient[1]);
    }
    float *p1 = p0 + (size_t)3 * n0 * K_pad * 4;
    for (int o = 0; o < 2; ++o) {
        float *p = o == 0 ? p0 : p1;
        st = bf16 ? vup_moments_tc(g, K, o, 3, p, s) : vup_moments_simt(g, K, o, 3, p, s);
        if (st != VUP_OK) return st;
    }
    return vup_ipsa_finish(g, K, (int)n0, (int)n1, grad_moments, dmu, dsigma, s);
}

extern "C" vup_status vup_propagate_ipsa(vup_grid g, const vup_densities *d, vup_precision precision,
                                         double *moments_raw, double *moments_central, float *hist,
                                         const double *grad_moments, float *dmu, float *dsigma,
                                         vup_stream_t stream) {
    if (!g || !dmu || !dsigma) return VUP_ERR_INVALID_ARG;
    vup_status st = vup_check_dens(g, d);
    if (st != VUP_OK) return st;
    if (precision < VUP_FP64 || precision > VUP_TF32X3) return VUP_ERR_INVALID_ARG;
    if (!g->have_model) return VUP_ERR_STATE;
    if (g->ndim == 2 && (precision == VUP_FP32 || precision == VUP_BF16X3)) {
        const IpsaOut ip{grad_moments, dmu, dsigma};
        return propagate_nd(g, d, precision, moments_raw, moments_central, hist, (cudaStream_t)stream, &ip);
    }
    if ((st = vup_propagate(g, d, precision, moments_raw, moments_central, hist, stream)) != VUP_OK) return st;
    return vup_ipsa_sensitivity(g, d, precision, grad_moments, dmu, dsigma, stream);
}

extern "C" vup_status vup_sync(vup_grid g, vup_stream_t stream) {
    if (!g) return VUP_ERR_INVALID_ARG;
    VUP_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int code = 0;
    VUP_CHECK_CUDA(cudaMemcpy(&code, g->dstatus, sizeof(int), cudaMemcpyDeviceToHost));
    if (code) VUP_CHECK_CUDA(cudaMemset(g->dstatus, 0, sizeof(int)));
    switch (code) {
    case 0: return VUP_OK;
    case VUP_DSTAT_EMPTY: return VUP_ERR_EMPTY_SUPPORT;
    case VUP_DSTAT_TIMEOUT: return VUP_ERR_TIMEOUT;
    case VUP_DSTAT_BOUNDS: return VUP_ERR_BOUNDS;
    default: return VUP_ERR_INVALID_ARG;
    }
}

extern "C" vup_status vup_grid_info(vup_grid g, vup_grid_info_t *info) {
    if (!g || !info) return VUP_ERR_INVALID_ARG;
    memset(info, 0, sizeof(*info));
    info->ndim = g->ndim;
    for (int d = 0; d < 3; ++d) info->n[d] = d < g->ndim ? g->n[d] : 1;
    info->N = g->N;
    info->n_bins = g->B;
    info->n_moments = g->J;
    info->have_model = g->have_model;
    if (g->have_model) {
        unsigned long long k[2];
        double sc[kScaleSlots] = {1.0, 0.0, 1.0};
        VUP_CHECK_CUDA(cudaDeviceSynchronize());
        VUP_CHECK_CUDA(cudaMemcpy(k, g->ext, sizeof(k), cudaMemcpyDeviceToHost));
        VUP_CHECK_CUDA(cudaMemcpy(sc, g->ydev_scale, sizeof(sc), cudaMemcpyDeviceToHost));
        auto inv = [](unsigned long long key) {
            unsigned long long u = (key >> 63) ? (key & 0x7fffffffffffffffull) : ~key;
            double v;
            memcpy(&v, &u, sizeof(v));
            return v;
        };
        info->ymin = inv(k[0]);
        info->ymax = inv(k[1]);
        info->yscale = sc[kScaleS];
        info->yshift = sc[kScaleC];
        if (g->ndim >= 2) {
            if (!g->layout_valid) {
                vup_status st = vup_build_layout(g, 0);
                if (st != VUP_OK) return st;
                VUP_CHECK_CUDA(cudaDeviceSynchronize());
            }
            int32_t sel[2] = {0, 0}, nr = 0, ni = 0, nrec = 0;
            VUP_CHECK_CUDA(cudaMemcpy(sel, g->hist_sel, sizeof(sel), cudaMemcpyDeviceToHost));
            const auto &HL = g->hl[0];  // the built layout's arrays
            VUP_CHECK_CUDA(cudaMemcpy(&nr, HL.n_runs, sizeof(int32_t), cudaMemcpyDeviceToHost));
            VUP_CHECK_CUDA(cudaMemcpy(&ni, HL.n_iv, sizeof(int32_t), cudaMemcpyDeviceToHost));
            VUP_CHECK_CUDA(cudaMemcpy(&nrec, HL.n_rec, sizeof(int32_t), cudaMemcpyDeviceToHost));
            info->hist_layout = sel[0];
            info->hist_stream = sel[1];
            info->hist_runs = nr;
            info->hist_intervals = ni;
            info->hist_records = nrec;
        }
    }
    return VUP_OK;
}

extern "C" vup_status vup_set_hist_stream(vup_grid g, int32_t stream_kind, vup_stream_t stream) {
    if (!g || g->ndim < 2 || stream_kind < -1 || stream_kind > 2) return VUP_ERR_INVALID_ARG;
    // the layout is rebuilt on next use with the choice (a forced point or
    // interval stream needs the key-sorted streams a record choice skips)
    if (stream_kind != g->hist_force) g->layout_valid = g->ndim == 1;
    g->hist_force = stream_kind;
    return VUP_OK;
}

extern "C" vup_status vup_set_weights_form(vup_grid g, int32_t form) {
    if (!g || form < -1 || form > 2) return VUP_ERR_INVALID_ARG;
    g->weights_form = form;
    return VUP_OK;
}

extern "C" vup_status vup_grid_copy(vup_grid g, int which, void *dst_dev, size_t nbytes, vup_stream_t stream) {
    if (!g || !dst_dev) return VUP_ERR_INVALID_ARG;
    if (!g->have_model) return VUP_ERR_STATE;
    const void *src = nullptr;
    size_t need = 0;
    switch (which) {
    case 0: src = g->y; need = sizeof(double) * g->N; break;
    case 1: src = g->bins; need = sizeof(int32_t) * g->N; break;
    case 2: {
        vup_status st = vup_natural_sort(g, (cudaStream_t)stream);
        if (st != VUP_OK) return st;
        src = g->perm;
        need = sizeof(int32_t) * g->N;
        break;
    }
    case 3: {
        // bin offsets of the stable sort by bin (built with it on 2-D / 3-D grids)
        vup_status st = vup_natural_sort(g, (cudaStream_t)stream);
        if (st != VUP_OK) return st;
        src = g->offsets;
        need = sizeof(int32_t) * (g->B + 1);
        break;
    }
    default: return VUP_ERR_INVALID_ARG;
    }
    if (nbytes != need) return VUP_ERR_INVALID_ARG;
    VUP_CHECK_CUDA(cudaMemcpyAsync(dst_dev, src, need, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return VUP_OK;
}
