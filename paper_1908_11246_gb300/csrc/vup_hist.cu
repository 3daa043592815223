// Output probability vectors (Eq. 4 / Eq. 5, Eq. VUP): H[k, b] = sum of the
// normalised input probabilities of the grid points whose model value falls in
// bin b.  The one-hot model matrix of Eq. MUP is applied as a segmented
// reduction over the grid points pre-sorted by bin ("sort and sum").
//
// Layout: lanes of a warp are 32 densities k; every lane walks the same
// sorted point stream, so control flow is uniform and the factor gathers hit
// 32 consecutive shared-memory words (conflict-free).  Points are grouped in
// runs that share the bin and every axis index but the last: inside a run
// only the last-axis factor is gathered (from shared memory); the product
// with the other axes' factors is applied once per run.  Each warp owns a
// chunk of runs; bins cut by chunk boundaries are written as partials and
// summed by a deterministic fix-up kernel.
#include "vup_internal.cuh"

#include <algorithm>

namespace {

constexpr int kHistWarps = 16;
constexpr int kKT = 32;              // densities per k-tile (one per lane)

struct HistArgs {
    const uint32_t *hpt;
    const int32_t *run_start, *run_rest, *run_bin;
    const int32_t *chunk_pt, *chunk_run, *chunk_bin;
    const int32_t *offsets;
    const float *g_last;      // factor table of the last axis  [n_last][K_pad]
    const float *g0, *g1;     // rest-axis factor tables (g1 only for 3-D)
    int64_t n1;               // size of axis 1 (3-D rest split)
    const DensStats *ds;
    int ndim;
    int64_t K, K_pad;
    int64_t n_last;
    int B;
    int C;                    // chunks per k-tile
    float *hist;              // [K][B]
    float *part;              // [C][2][K_pad]
};

constexpr int kPF = 16;              // runs whose rest-axis factor is prefetched ahead

template <bool kSmem>
__global__ void __launch_bounds__(kHistWarps * 32, 1) k_hist(HistArgs A) {
    extern __shared__ __align__(16) float ws[];  // [n_last][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t kt = blockIdx.y;
    const int64_t k0 = kt * kKT;
    const int64_t k = k0 + lane;
    if (kSmem) {
        for (int64_t e = threadIdx.x; e < A.n_last * kKT; e += blockDim.x)
            ws[e] = A.g_last[(e >> 5) * A.K_pad + k0 + (e & 31)];
        __syncthreads();
    }
    const float *wl = kSmem ? ws + lane : A.g_last + k;
    const int64_t wstride = kSmem ? kKT : A.K_pad;

    float invZ = 0.f;
    if (k < A.K) {
        double z = 1.0;
        for (int d = 0; d < A.ndim; ++d) z *= A.ds[k * A.ndim + d].invZ;
        invZ = (float)z;
    }
    const int c = blockIdx.x * kHistWarps + warp;
    if (c >= A.C) return;
    const int32_t p0 = A.chunk_pt[c], p1 = A.chunk_pt[c + 1];
    if (p0 >= p1) return;
    const int32_t r0 = A.chunk_run[c], r1 = A.chunk_run[c + 1];
    const int32_t first_bin = A.chunk_bin[2 * c];

    // rest-axis factor of run r for this lane's density
    auto wrest = [&](int32_t r) -> float {
        if (r >= r1) return 0.f;
        const int32_t rest = A.run_rest[r];
        if (A.ndim == 3) {
            const int64_t a0 = rest / A.n1, a1 = rest - a0 * A.n1;
            return A.g0[a0 * A.K_pad + k] * A.g1[a1 * A.K_pad + k];
        }
        return A.g0[(int64_t)rest * A.K_pad + k];
    };
    auto flush_bin = [&](int32_t b, float v) {
        const float val = v * invZ;
        const bool shared = A.offsets[b] < p0 || A.offsets[b + 1] > p1;
        if (shared) {
            const int side = (b == first_bin) ? 0 : 1;
            A.part[((int64_t)c * 2 + side) * A.K_pad + k] = val;
        } else if (k < A.K) {
            A.hist[k * A.B + b] = val;
        }
    };

    int32_t cur_bin = A.run_bin[r0];
    float bacc = 0.f;
    float wa[kPF], wb[kPF];
#pragma unroll
    for (int u = 0; u < kPF; ++u) wa[u] = wrest(r0 + u);

    // one block of kPF runs: sum the last-axis factors of each run's points,
    // scale by the run's rest factor, flush at bin changes
    auto do_block = [&](int32_t rb, const float (&w)[kPF]) {
#pragma unroll
        for (int u = 0; u < kPF; ++u) {
            const int32_t r = rb + u;
            if (r >= r1) break;
            const int32_t s0 = A.run_start[r], s1 = A.run_start[r + 1];
            float acc = 0.f;
            int32_t p = s0;
            for (; p + 2 <= s1; p += 2) {
                const uint32_t u0 = A.hpt[p], u1 = A.hpt[p + 1];
                const float v0 = wl[(int64_t)(u0 & 0xffffu) * wstride];
                const float v1 = wl[(int64_t)(u1 & 0xffffu) * wstride];
                acc += v0;
                acc += v1;
            }
            if (p < s1) acc += wl[(int64_t)(A.hpt[p] & 0xffffu) * wstride];
            bacc = fmaf(w[u], acc, bacc);
            const int32_t nb = r + 1 < r1 ? A.run_bin[r + 1] : -1;
            if (nb != cur_bin) {
                flush_bin(cur_bin, bacc);
                bacc = 0.f;
                cur_bin = nb;
            }
        }
    };
    for (int32_t rb = r0; rb < r1; rb += 2 * kPF) {
#pragma unroll
        for (int u = 0; u < kPF; ++u) wb[u] = wrest(rb + kPF + u);
        do_block(rb, wa);
        if (rb + kPF >= r1) break;
#pragma unroll
        for (int u = 0; u < kPF; ++u) wa[u] = wrest(rb + 2 * kPF + u);
        do_block(rb + kPF, wb);
    }
}

__device__ __forceinline__ int chunk_of(const int32_t *chunk_pt, int C, int32_t p) {
    int lo = 0, hi = C;  // last c with chunk_pt[c] <= p
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (chunk_pt[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Bins cut by chunk boundaries: sum the partials of every chunk overlapping
// the bin (in chunk order); empty bins are zero.
__global__ void k_hist_fixup(const int32_t *__restrict__ offsets, const int32_t *__restrict__ chunk_pt,
                             const int32_t *__restrict__ chunk_bin, const float *__restrict__ part, int C,
                             int64_t K, int64_t K_pad, int B, float *__restrict__ hist) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (k >= K) return;
    const int32_t o0 = offsets[b], o1 = offsets[b + 1];
    if (o0 == o1) {
        hist[k * B + b] = 0.f;
        return;
    }
    const int c0 = chunk_of(chunk_pt, C, o0), c1 = chunk_of(chunk_pt, C, o1 - 1);
    if (c0 == c1) return;  // written directly by its chunk
    float s = 0.f;
    for (int c = c0; c <= c1; ++c) {
        if (chunk_pt[c] >= chunk_pt[c + 1]) continue;
        const int side = chunk_bin[2 * c] == b ? 0 : 1;
        s += part[((int64_t)c * 2 + side) * K_pad + k];
    }
    hist[k * B + b] = s;
}

}  // namespace

int vup_hist_chunks_for(int64_t N) {
    int64_t S = N / ((int64_t)kHistWarps * 16384);
    S = std::max<int64_t>(1, std::min<int64_t>(16, S));
    return (int)(S * kHistWarps);
}

vup_status vup_hist_fused(vup_grid g, int64_t K, float *hist, cudaStream_t s) {
    const int64_t K_pad = ceil_div64(K, 128) * 128;
    HistArgs A{};
    A.hpt = g->hpt;
    A.run_start = g->run_start;
    A.run_rest = g->run_rest;
    A.run_bin = g->run_bin;
    A.chunk_pt = g->chunk_pt;
    A.chunk_run = g->chunk_run;
    A.chunk_bin = g->chunk_bin;
    A.offsets = g->offsets;
    const int nd = g->ndim;
    auto tab = [&](int axis) {
        int64_t off = 0;
        for (int q = 0; q < axis; ++q) off += g->n[q] * K_pad;
        return (const float *)g->ftab.p + off;
    };
    A.g_last = tab(nd - 1);
    A.g0 = tab(0);
    A.g1 = nd == 3 ? tab(1) : nullptr;
    A.n1 = g->n[1];
    A.ds = (const DensStats *)g->dstats.p;
    A.ndim = nd;
    A.K = K;
    A.K_pad = K_pad;
    A.n_last = g->n[nd - 1];
    A.B = g->B;
    A.C = g->n_chunks;
    A.hist = hist;
    A.part = (float *)g->hist_part.p;
    const size_t smem = sizeof(float) * (size_t)A.n_last * kKT;
    dim3 grd((unsigned)(A.C / kHistWarps), (unsigned)ceil_div64(K, kKT));
    {
    VUP_PROF("hist_segmented", s, 1);
    if (smem <= 200 * 1024) {
        static bool attr_set = false;
        if (!attr_set) {
            VUP_CHECK_CUDA(cudaFuncSetAttribute(k_hist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                200 * 1024));
            attr_set = true;
        }
        k_hist<true><<<grd, kHistWarps * 32, smem, s>>>(A);
    } else {
        k_hist<false><<<grd, kHistWarps * 32, 0, s>>>(A);
    }
    VUP_CHECK_LAUNCH();
    }
    VUP_PROF("hist_fixup", s, 1);
    dim3 fg((unsigned)ceil_div64(K, 128), (unsigned)g->B);
    k_hist_fixup<<<fg, 128, 0, s>>>(g->offsets, g->chunk_pt, g->chunk_bin, (const float *)g->hist_part.p, A.C, K,
                                    K_pad, g->B, hist);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}
