// Batched uneven propagation: many independent 2-D instances (each with its
// own grid, model outputs, densities and outputs, sizes varying by orders of
// magnitude) run stage by stage, every stage one launch over the work items
// of all instances, longest items first:
//
//   density prep  ->  moment contraction (tcgen05 or FP32 SIMT)  ->  FP64
//   finish  ->  segmented histogram  ->  histogram finish
//
// The launch sequence of a batch (same grids, densities and outputs) is
// captured once into a CUDA graph and replayed on later calls.  For the
// tensor-core contraction the tile width of each instance is capped by a
// per-batch-shape choice that the first call makes by timing the candidates
// (caps 256, 128, 64); the choice is kept in memory and, when the environment
// variable VUP_TUNE_CACHE names a file, appended to it as one JSON object per
// line and read back by later processes.
#include "vup_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace {

struct Stages {
    void *dens = nullptr, *tc = nullptr, *simt = nullptr, *fin = nullptr, *hist = nullptr;
};

void free_stages(Stages &S) {
    vup_density_plan_free(S.dens);
    vup_tc_plan_free(S.tc);
    vup_simt_plan_free(S.simt);
    vup_finish_plan_free(S.fin);
    vup_hist_plan_free(S.hist);
    S = Stages();
}

struct Entry {
    std::vector<uint64_t> key;
    int device = 0;
    bool bf16 = false;
    int bn_cap = 0;
    int *dstatus = nullptr;
    Stages st;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;
};

void free_entry(Entry *e) {
    if (!e) return;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    free_stages(e->st);
    delete e;
}

constexpr size_t kMaxEntries = 8;
std::mutex g_mu;
std::vector<Entry *> g_entries;
uint64_t g_clock = 0;
std::map<std::string, int> g_tuned;  // batch shape -> tile-width cap
bool g_tune_loaded = false;

thread_local int t_bn_cap = 0, t_source = -1;
thread_local double t_tune_ms = 0.0;

uint64_t fnv(uint64_t h, uint64_t v) {
    for (int i = 0; i < 8; ++i) {
        h ^= (v >> (8 * i)) & 0xff;
        h *= 1099511628211ull;
    }
    return h;
}

// Stage launches of one batch on stream s.
vup_status run_stages(const Entry &e, cudaStream_t s) {
    vup_status st;
    if (e.st.dens && (st = vup_density_batched(e.st.dens, s)) != VUP_OK) return st;
    if (e.st.tc && (st = vup_tc_batched(e.st.tc, e.dstatus, s)) != VUP_OK) return st;
    if (e.st.simt && (st = vup_simt_batched(e.st.simt, s)) != VUP_OK) return st;
    if (e.st.fin && (st = vup_finish_batched(e.st.fin, s)) != VUP_OK) return st;
    if (e.st.hist && (st = vup_hist_batched(e.st.hist, s)) != VUP_OK) return st;
    return VUP_OK;
}

vup_status build_stages(int n, const vup_grid *g, const vup_densities *d, bool bf16, int bn_cap,
                        double *const *raws, float *const *hists, Stages &S) {
    std::vector<vup_grid> mg;
    std::vector<int64_t> mK, nct;
    std::vector<float *> parts;
    std::vector<double *> mraw;
    std::vector<int> bns;
    for (int i = 0; i < n; ++i) {
        if (!raws || !raws[i]) continue;
        const Orient &o = g[i]->orient[0];
        mg.push_back(g[i]);
        mK.push_back(d[i].K);
        parts.push_back((float *)g[i]->partials.p);
        mraw.push_back(raws[i]);
        const int bn = bf16 ? vup_tc_bn_for(o, bn_cap) : 0;
        bns.push_back(bn);
        nct.push_back(bf16 ? vup_tc_col_tiles_bn(o, bn) : vup_simt_col_tiles(o));
    }
    bool any_h = false;
    for (int i = 0; i < n; ++i) any_h |= hists && hists[i];
    if (mg.empty() && !any_h) return VUP_OK;
    vup_status st;
    if ((st = vup_density_plan(n, g, d, bf16 && !mg.empty(), &S.dens)) != VUP_OK) return st;
    const int m = (int)mg.size();
    if (m) {
        st = bf16 ? vup_tc_plan(m, mg.data(), mK.data(), bns.data(), parts.data(), &S.tc)
                  : vup_simt_plan(m, mg.data(), mK.data(), parts.data(), &S.simt);
        if (st != VUP_OK) return st;
        if ((st = vup_finish_plan(m, mg.data(), mK.data(), nct.data(), parts.data(), mraw.data(), nullptr,
                                  &S.fin)) != VUP_OK)
            return st;
    }
    if (any_h) {
        std::vector<int64_t> K(n);
        for (int i = 0; i < n; ++i) K[i] = d[i].K;
        if ((st = vup_hist_plan(n, g, K.data(), hists, &S.hist)) != VUP_OK) return st;
    }
    return VUP_OK;
}

vup_status capture(Entry &e) {
    cudaStream_t cs;
    VUP_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return VUP_ERR_CUDA;
    }
    const vup_status st = run_stages(e, cs);
    cudaGraph_t gr = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &gr);
    cudaStreamDestroy(cs);
    if (st != VUP_OK || ce != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return st != VUP_OK ? st : VUP_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&e.exec, gr, 0) != cudaSuccess) {
        cudaGraphDestroy(gr);
        e.exec = nullptr;
        return VUP_ERR_CUDA;
    }
    e.graph = gr;
    return VUP_OK;
}

// Mean device time of `reps` replays after one warm-up replay.
double time_graph(cudaGraphExec_t ex, cudaStream_t s, int reps) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return 1e30;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return 1e30;
    }
    float ms = 1e30f;
    if (cudaGraphLaunch(ex, s) == cudaSuccess && cudaEventRecord(a, s) == cudaSuccess) {
        bool ok = true;
        for (int r = 0; r < reps && ok; ++r) ok = cudaGraphLaunch(ex, s) == cudaSuccess;
        if (ok && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess)
            cudaEventElapsedTime(&ms, a, b);
        else
            ms = 1e30f;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return (double)ms / reps;
}

void load_tune_file() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("VUP_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char shape[64];
        int cap;
        if (sscanf(line, " {\"shape\": \"%63[0-9a-f]\", \"bn_cap\": %d", shape, &cap) == 2 &&
            (cap == 64 || cap == 128 || cap == 256))
            g_tuned[shape] = cap;
    }
    fclose(f);
}

void store_tune(const std::string &shape, int cap, const double *ms, const int *caps, int n_c) {
    g_tuned[shape] = cap;
    const char *path = getenv("VUP_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "{\"shape\": \"%s\", \"bn_cap\": %d, \"ms\": {", shape.c_str(), cap);
    for (int c = 0; c < n_c; ++c) fprintf(f, "%s\"%d\": %.6f", c ? ", " : "", caps[c], ms[c]);
    fprintf(f, "}}\n");
    fclose(f);
}

}  // namespace

extern "C" vup_status vup_propagate_batched(int n_inst, const vup_grid *g, const vup_densities *d,
                                            vup_precision precision, double *const *moments_raw,
                                            float *const *hist, vup_stream_t stream) {
    if (n_inst < 0 || (n_inst > 0 && (!g || !d))) return VUP_ERR_INVALID_ARG;
    if (precision < VUP_FP64 || precision > VUP_TF32X3) return VUP_ERR_INVALID_ARG;
    if (precision != VUP_FP32 && precision != VUP_BF16X3) return VUP_ERR_UNSUPPORTED;
    if (n_inst == 0) return VUP_OK;
    const bool bf16 = precision == VUP_BF16X3;
    for (int i = 0; i < n_inst; ++i) {
        if (!g[i]) return VUP_ERR_INVALID_ARG;
        vup_status st = vup_check_dens(g[i], &d[i]);
        if (st != VUP_OK) return st;
        if (g[i]->ndim != 2 || !vup_hist_batchable(g[i])) return VUP_ERR_UNSUPPORTED;
        if (!g[i]->have_model) return VUP_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    VUP_CHECK_CUDA(cudaStreamIsCapturing(s, &cst));
    const bool capturing = cst != cudaStreamCaptureStatusNone;
    int dev = 0;
    VUP_CHECK_CUDA(cudaGetDevice(&dev));

    std::lock_guard<std::mutex> lk(g_mu);
    if (!capturing) {
        // scratch for the largest work any plan of this batch may need
        for (int i = 0; i < n_inst; ++i) {
            const int64_t K = d[i].K, K_pad = ceil_div64(K, 128) * 128;
            vup_status st;
            if ((st = vup_reserve_k(g[i], K, bf16, false)) != VUP_OK) return st;
            if ((st = vup_build_tables(g[i], kOrientLast, bf16 ? 1 : 0, s)) != VUP_OK) return st;
            if (hist && hist[i] && (st = vup_ensure_layout(g[i], s)) != VUP_OK) return st;
            if ((st = vup_density_reserve(g[i], K)) != VUP_OK) return st;
            if (bf16 &&
                (st = devbuf_reserve(g[i]->partials,
                                     sizeof(float) * 4 * K_pad * vup_tc_col_tiles_bn(g[i]->orient[0], 64))) != VUP_OK)
                return st;
        }
    }
    std::vector<uint64_t> key;
    key.reserve(4 + (size_t)n_inst * 20);
    key.push_back((uint64_t)dev);
    key.push_back((uint64_t)precision);
    key.push_back((uint64_t)n_inst);
    for (int i = 0; i < n_inst; ++i) {
        const vup_grid G = g[i];
        const vup_densities &D = d[i];
        const uint64_t w[] = {(uint64_t)G, G->model_gen, (uint64_t)D.K, (uint64_t)D.kind, (uint64_t)D.mu,
                              (uint64_t)D.sigma, (uint64_t)D.lo, (uint64_t)D.hi,
                              (uint64_t)(moments_raw ? moments_raw[i] : nullptr),
                              (uint64_t)(hist ? hist[i] : nullptr), (uint64_t)G->ftab.p, (uint64_t)G->dstats.p,
                              (uint64_t)G->dconst.p, (uint64_t)G->dpart.p, (uint64_t)G->partials.p,
                              (uint64_t)G->atab_hi.p, (uint64_t)G->atab_lo.p, (uint64_t)G->hist_part.p,
                              (uint64_t)G->hist_direct.p};
        key.insert(key.end(), std::begin(w), std::end(w));
    }
    Entry *e = nullptr;
    for (Entry *x : g_entries)
        if (x->key == key) e = x;

    if (!e) {
        if (capturing) return VUP_ERR_STATE;  // plans are built (and tuned) by an uncaptured first call
        // batch shape (sizes only) for the tuning decision
        uint64_t h = 1469598103934665603ull;
        h = fnv(h, (uint64_t)precision);
        for (int i = 0; i < n_inst; ++i) {
            h = fnv(h, (uint64_t)g[i]->n[0]);
            h = fnv(h, (uint64_t)g[i]->n[1]);
            h = fnv(h, (uint64_t)d[i].K);
            h = fnv(h, (uint64_t)g[i]->B);
            h = fnv(h, (uint64_t)g[i]->J);
            h = fnv(h, (uint64_t)((moments_raw && moments_raw[i]) ? 1 : 0) | ((hist && hist[i]) ? 2 : 0));
        }
        char shape[32];
        snprintf(shape, sizeof shape, "%016llx", (unsigned long long)h);
        load_tune_file();
        std::vector<int> caps;
        int source = 1;
        if (!bf16) {
            caps = {0};
        } else {
            auto it = g_tuned.find(shape);
            if (it != g_tuned.end()) {
                caps = {it->second};
            } else {
                caps = {256, 128, 64};
                source = 2;
            }
        }
        // evict the least recently used plan (its graph may still be in flight)
        if (g_entries.size() >= kMaxEntries) {
            auto lru = std::min_element(g_entries.begin(), g_entries.end(),
                                        [](const Entry *a, const Entry *b) { return a->used < b->used; });
            VUP_CHECK_CUDA(cudaDeviceSynchronize());
            free_entry(*lru);
            g_entries.erase(lru);
        }
        std::vector<Entry *> cand;
        std::vector<double> ms;
        vup_status st = VUP_OK;
        for (int cap : caps) {
            Entry *c = new Entry();
            c->key = key;
            c->device = dev;
            c->bf16 = bf16;
            c->bn_cap = cap;
            c->dstatus = g[0]->dstatus;
            st = build_stages(n_inst, g, d, bf16, cap, moments_raw, hist, c->st);
            if (st == VUP_OK) st = capture(*c);
            if (st != VUP_OK) {
                free_entry(c);
                break;
            }
            cand.push_back(c);
            ms.push_back(caps.size() > 1 ? time_graph(c->exec, s, 3) : 0.0);
        }
        if (st != VUP_OK) {
            if (!cand.empty()) cudaStreamSynchronize(s);
            for (Entry *c : cand) free_entry(c);
            return st;
        }
        size_t best = 0;
        for (size_t c = 1; c < cand.size(); ++c)
            if (ms[c] < ms[best]) best = c;
        if (cand.size() > 1) {
            VUP_CHECK_CUDA(cudaStreamSynchronize(s));
            store_tune(shape, caps[best], ms.data(), caps.data(), (int)caps.size());
            t_tune_ms = 0;
            for (double x : ms) t_tune_ms += 4 * x;
        } else {
            t_tune_ms = 0;
        }
        for (size_t c = 0; c < cand.size(); ++c)
            if (c != best) free_entry(cand[c]);
        e = cand[best];
        g_entries.push_back(e);
        t_source = source;
    } else {
        t_source = 0;
        t_tune_ms = 0;
    }
    e->used = ++g_clock;
    t_bn_cap = e->bn_cap;
    // inside a caller's capture the stage kernels join the caller's graph; with
    // profiling on they run one by one so that each stage is timed
    if (capturing || vup_profiling()) return run_stages(*e, s);
    VUP_CHECK_CUDA(cudaGraphLaunch(e->exec, s));
    return VUP_OK;
}

extern "C" vup_status vup_batched_report(int *bn_cap, int *source, double *tune_ms) {
    if (!bn_cap || !source || !tune_ms) return VUP_ERR_INVALID_ARG;
    *bn_cap = t_bn_cap;
    *source = t_source;
    *tune_ms = t_tune_ms;
    return VUP_OK;
}
