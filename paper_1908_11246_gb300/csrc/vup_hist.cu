// Output probability vectors (Eq. 4 / Eq. 5, Eq. VUP): H[k, b] = sum of the
// normalised input probabilities of the grid points whose model value falls in
// bin b.  The one-hot model matrix of Eq. MUP is applied as a segmented
// reduction over the grid points pre-sorted by bin ("sort and sum").
//
// Layout: lanes of a warp are 32 densities k; every lane walks the same
// sorted point stream, so control flow is uniform and the factor gathers hit
// 32 consecutive shared-memory words (conflict-free).  Points are grouped in
// runs that share the bin and every axis index but the gathered ("last")
// one: inside a run only the last-axis factor is gathered, from a shared-
// memory tile; the product with the other axes' factors is applied once per
// run.  Those factors are loaded four runs ahead: the run-end word of run r
// carries the rest index of run r + 4.  The point stream is staged into
// shared memory with bulk asynchronous copies (cp.async.bulk + mbarrier) and
// read four points per broadcast load.  Each warp owns a chunk of runs; bins
// cut by chunk boundaries are written as partials and summed by a
// deterministic fix-up kernel.  On 2-D grids two layouts exist (either axis
// gathered); the device uses the one with fewer runs.
#include "vup_internal.cuh"

#include <algorithm>

namespace {

constexpr int kHistWarps = 32;
constexpr int kKT = 32;                      // densities per k-tile (one per lane)
constexpr int kWin = 128;                    // sorted-point words per staging buffer
constexpr uint32_t kOffMask = 0x7fffu << 7;  // gathered-axis row byte offset (index << 7)
constexpr uint32_t kRunEnd = 1u << 30, kBinEnd = 1u << 31;
constexpr uint32_t kFlags = kRunEnd | kBinEnd;
constexpr uint32_t kSpin = 1u << 26;
constexpr int kPF = 16;                      // runs prefetched per block (global fallback)

struct LayoutArgs {
    const uint32_t *hpt;
    const int32_t *run_start, *run_rest, *run_bin;
    const int32_t *chunk_pt, *chunk_run, *chunk_bin;
    const float *g_last;  // factor table of the gathered axis  [n_last][K_pad]
    const float *g0, *g1; // rest-axis factor tables (g1 only for 3-D)
    int64_t n_last;
    int64_t n1;           // size of the second rest axis (3-D)
};

struct HistArgs {
    LayoutArgs L0, L1;
    const int32_t *sel;   // device: chosen layout
    const int32_t *offsets;
    const DensStats *ds;
    int ndim;
    int64_t K, K_pad;
    int B;
    int C;                // chunks per k-tile
    float *hist;          // [K][B]
    float *part;          // [C][2][K_pad]
    int *dstatus;
};

__device__ __forceinline__ LayoutArgs pick(const HistArgs &A) { return A.sel[0] ? A.L1 : A.L0; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// completing on `bar`.
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Shared memory of k_hist_smem: the gathered-axis factor tile [n_last + 1][32]
// (the extra row is zero; foreign points of a chunk's first and last group
// point at it), per warp 2 staging buffers of kWin point words, 2 mbarriers
// per warp.
__host__ __device__ inline size_t hist_tile_bytes(int64_t n_last) { return (size_t)((n_last + 1) * 128); }
__host__ __device__ inline size_t hist_warp_bytes() { return (size_t)2 * kWin * 4; }
__host__ __device__ inline size_t hist_smem_bytes(int64_t n_last) {
    return hist_tile_bytes(n_last) + kHistWarps * hist_warp_bytes() + kHistWarps * 2 * sizeof(uint64_t);
}

template <int NF>
__global__ void __launch_bounds__(kHistWarps * 32, 1) k_hist_smem(HistArgs A, int64_t n_tile_rows) {
    extern __shared__ __align__(128) uint8_t sm[];
    const LayoutArgs H = pick(A);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k0 = (int64_t)blockIdx.y * kKT;
    const int64_t k = k0 + lane;
    float *ws = reinterpret_cast<float *>(sm);
    const size_t tb = hist_tile_bytes(n_tile_rows);
    uint32_t *win = reinterpret_cast<uint32_t *>(sm + tb + (size_t)warp * hist_warp_bytes());
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + tb + kHistWarps * hist_warp_bytes()) + 2 * warp;

    // gathered-axis factor tile of this k-tile (16-byte asynchronous copies) + zero row
    for (int64_t e = threadIdx.x; e < H.n_last * 8; e += blockDim.x) {
        const int64_t a = e >> 3, c = e & 7;
        cp_async16(ws + a * 32 + c * 4, H.g_last + a * A.K_pad + k0 + c * 4);
    }
    cp_async_commit();
    if (threadIdx.x < 32) ws[H.n_last * 32 + threadIdx.x] = 0.f;
    cp_async_wait_all();
    __syncthreads();

    const int c = blockIdx.x * kHistWarps + warp;
    if (c >= A.C) return;
    const int32_t p0 = H.chunk_pt[c], p1 = H.chunk_pt[c + 1];
    if (p0 >= p1) return;
    const int32_t r0 = H.chunk_run[c], r1 = H.chunk_run[c + 1];
    const int32_t first_bin = H.chunk_bin[2 * c];
    float invZ = 0.f;
    if (k < A.K) {
        double z = 1.0;
        for (int d = 0; d < A.ndim; ++d) z *= A.ds[k * A.ndim + d].invZ;
        invZ = (float)z;
    }

    // staging of the sorted point stream: buffer b holds window wi (wi & 1 == b)
    const int32_t wb0 = p0 & ~(kWin - 1);
    if (lane == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        bulk_copy(win, H.hpt + wb0, kWin * 4, &mbar[0]);
        if (wb0 + kWin < p1) bulk_copy(win + kWin, H.hpt + wb0 + kWin, kWin * 4, &mbar[1]);
    }
    __syncwarp();

    // rest-axis factors of runs r .. r + 3, rotated through registers
    const float *g0k = H.g0 + k;
    const float *g1k = NF == 2 ? H.g1 + k : nullptr;
    const int64_t K_pad = A.K_pad;
    auto rest_factor = [&](int32_t r) -> float {
        if (r >= r1) return 0.f;
        const int32_t rest = H.run_rest[r];
        if (NF == 2) {
            const int32_t a0 = rest / (int32_t)H.n1, a1 = rest - a0 * (int32_t)H.n1;
            return g0k[a0 * K_pad] * g1k[a1 * K_pad];
        }
        return g0k[rest * K_pad];
    };
    float f0 = rest_factor(r0), f1 = rest_factor(r0 + 1), f2 = rest_factor(r0 + 2), f3 = rest_factor(r0 + 3);
    // factor of run r + 4, decoded from run r's end word (the load stays in flight)
    auto coded_factor = [&](uint32_t u) -> float {
        if (NF == 2) {
            const uint32_t a0 = u & 0x7fu, a1 = (u >> 22) & 0xffu;
            return g0k[(int64_t)a0 * K_pad] * g1k[(int64_t)a1 * K_pad];
        }
        const uint32_t idx = (u & 0x7fu) | ((u >> 15) & 0x7f80u);
        return g0k[(int64_t)idx * K_pad];
    };

    int32_t r = r0, cur_bin = H.run_bin[r0];
    float acc = 0.f, bacc = 0.f;
    const uint32_t wsl = smem_u32(ws) + lane * 4;
    const uint32_t null_word = (uint32_t)H.n_last << 7;  // zero row, no flags

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
    auto run_end = [&](uint32_t u) {
        bacc = fmaf(f0, acc, bacc);
        acc = 0.f;
        if (u & kBinEnd) {
            flush_bin(cur_bin, bacc);
            bacc = 0.f;
            cur_bin = r + 1 < r1 ? H.run_bin[r + 1] : -1;
        }
        ++r;
        f0 = f1;
        f1 = f2;
        f2 = f3;
        f3 = coded_factor(u);
    };
    auto gather = [&](uint32_t u) -> float {
        float v;
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(wsl + (u & kOffMask)));
        return v;
    };
    // words without flags carry nothing but the row byte offset (run codes sit
    // on run-end words only), so the common path needs no masking
    auto gather_raw = [&](uint32_t u) -> float {
        float v;
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(wsl + u));
        return v;
    };
    auto group = [&](const uint4 v) {
        if (((v.x | v.y | v.z | v.w) & kFlags) == 0) {
            const float a0 = gather_raw(v.x), a1 = gather_raw(v.y), a2 = gather_raw(v.z), a3 = gather_raw(v.w);
            acc += a0;
            acc += a1;
            acc += a2;
            acc += a3;
        } else {
            const float a0 = gather(v.x), a1 = gather(v.y), a2 = gather(v.z), a3 = gather(v.w);
            acc += a0;
            if (v.x & kFlags) run_end(v.x);
            acc += a1;
            if (v.y & kFlags) run_end(v.y);
            acc += a2;
            if (v.z & kFlags) run_end(v.z);
            acc += a3;
            if (v.w & kFlags) run_end(v.w);
        }
    };
    // a group cut by the chunk bounds: foreign points read the zero row
    auto masked = [&](uint4 v, int pa, int lo, int hi) {
        if (pa + 0 < lo || pa + 0 >= hi) v.x = null_word;
        if (pa + 1 < lo || pa + 1 >= hi) v.y = null_word;
        if (pa + 2 < lo || pa + 2 >= hi) v.z = null_word;
        if (pa + 3 < lo || pa + 3 >= hi) v.w = null_word;
        return v;
    };

    int wi = 0;
    for (int32_t wbase = wb0; wbase < p1; wbase += kWin, ++wi) {
        const int b = wi & 1;
        for (uint32_t i = 0; !mbar_try_wait(&mbar[b], (wi >> 1) & 1); ++i) {
            if (i > kSpin) {  // a staged copy never landed: record and stop
                atomicCAS(A.dstatus, 0, VUP_DSTAT_TIMEOUT);
                return;
            }
        }
        const uint32_t *wv = win + b * kWin;
        const int lo = (p0 > wbase ? p0 : wbase) - wbase;
        const int hi = (p1 < wbase + kWin ? p1 : wbase + kWin) - wbase;
        const int ga = (lo + 3) & ~3, gb = hi & ~3;   // whole groups [ga, gb)
        if (lo & 3) {
            const int pa = lo & ~3;
            group(masked(*reinterpret_cast<const uint4 *>(wv + pa), pa, lo, hi));
        }
#pragma unroll 2
        for (int pa = ga; pa < gb; pa += 4) group(*reinterpret_cast<const uint4 *>(wv + pa));
        if ((hi & 3) && gb >= ga) group(masked(*reinterpret_cast<const uint4 *>(wv + gb), gb, lo, hi));
        __syncwarp();
        if (lane == 0 && wbase + 2 * kWin < p1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bulk_copy(win + b * kWin, H.hpt + wbase + 2 * kWin, kWin * 4, &mbar[b]);
        }
    }
    if (cur_bin >= 0) flush_bin(cur_bin, bacc);
}

// Fallback for gathered axes too long for the shared-memory tile (or 3-D
// rest indices beyond the run-end encoding): factors are gathered from global
// memory (L1-cached), rest-axis factors prefetched in register blocks.
__global__ void __launch_bounds__(kHistWarps * 32, 1) k_hist_global(HistArgs A) {
    const LayoutArgs H = pick(A);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k0 = (int64_t)blockIdx.y * kKT;
    const int64_t k = k0 + lane;
    const float *wl = H.g_last + k;
    float invZ = 0.f;
    if (k < A.K) {
        double z = 1.0;
        for (int d = 0; d < A.ndim; ++d) z *= A.ds[k * A.ndim + d].invZ;
        invZ = (float)z;
    }
    const int c = blockIdx.x * kHistWarps + warp;
    if (c >= A.C) return;
    const int32_t p0 = H.chunk_pt[c], p1 = H.chunk_pt[c + 1];
    if (p0 >= p1) return;
    const int32_t r0 = H.chunk_run[c], r1 = H.chunk_run[c + 1];
    const int32_t first_bin = H.chunk_bin[2 * c];
    auto wrest = [&](int32_t r) -> float {
        if (r >= r1) return 0.f;
        const int32_t rest = H.run_rest[r];
        if (A.ndim == 3) {
            const int64_t a0 = rest / H.n1, a1 = rest - a0 * H.n1;
            return H.g0[a0 * A.K_pad + k] * H.g1[a1 * A.K_pad + k];
        }
        return H.g0[(int64_t)rest * A.K_pad + k];
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
    int32_t cur_bin = H.run_bin[r0];
    float bacc = 0.f;
    for (int32_t rb = r0; rb < r1; rb += kPF) {
        float w[kPF];
#pragma unroll
        for (int u = 0; u < kPF; ++u) w[u] = wrest(rb + u);
        for (int u = 0; u < kPF; ++u) {
            const int32_t r = rb + u;
            if (r >= r1) break;
            float acc = 0.f;
            for (int32_t p = H.run_start[r]; p < H.run_start[r + 1]; ++p)
                acc += wl[(int64_t)((H.hpt[p] & kOffMask) >> 7) * A.K_pad];
            bacc = fmaf(w[u], acc, bacc);
            const int32_t nb = r + 1 < r1 ? H.run_bin[r + 1] : -1;
            if (nb != cur_bin) {
                flush_bin(cur_bin, bacc);
                bacc = 0.f;
                cur_bin = nb;
            }
        }
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
__global__ void k_hist_fixup(HistArgs A) {
    const LayoutArgs H = pick(A);
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (k >= A.K) return;
    const int32_t o0 = A.offsets[b], o1 = A.offsets[b + 1];
    if (o0 == o1) {
        A.hist[k * A.B + b] = 0.f;
        return;
    }
    const int c0 = chunk_of(H.chunk_pt, A.C, o0), c1 = chunk_of(H.chunk_pt, A.C, o1 - 1);
    if (c0 == c1) return;  // written directly by its chunk
    float s = 0.f;
    for (int c = c0; c <= c1; ++c) {
        if (H.chunk_pt[c] >= H.chunk_pt[c + 1]) continue;
        const int side = H.chunk_bin[2 * c] == b ? 0 : 1;
        s += A.part[((int64_t)c * 2 + side) * A.K_pad + k];
    }
    A.hist[k * A.B + b] = s;
}

}  // namespace

int vup_hist_chunks_for(int64_t N) {
    int64_t S = N / ((int64_t)kHistWarps * 16384);
    S = std::max<int64_t>(1, std::min<int64_t>(16, S));
    return (int)(S * kHistWarps);
}

vup_status vup_hist_fused(vup_grid g, int64_t K, float *hist, cudaStream_t s) {
    const int64_t K_pad = ceil_div64(K, 128) * 128;
    const int nd = g->ndim;
    auto tab = [&](int axis) {
        int64_t off = 0;
        for (int q = 0; q < axis; ++q) off += g->n[q] * K_pad;
        return (const float *)g->ftab.p + off;
    };
    HistArgs A{};
    int64_t rows = 0;
    for (int l = 0; l < 2; ++l) {
        const auto &HL = g->hl[l < g->n_layouts ? l : 0];
        LayoutArgs &La = l == 0 ? A.L0 : A.L1;
        La.hpt = HL.hpt;
        La.run_start = HL.run_start;
        La.run_rest = HL.run_rest;
        La.run_bin = HL.run_bin;
        La.chunk_pt = HL.chunk_pt;
        La.chunk_run = HL.chunk_run;
        La.chunk_bin = HL.chunk_bin;
        La.g_last = tab(HL.last_axis);
        if (nd == 3) {
            La.g0 = tab(0);
            La.g1 = tab(1);
            La.n1 = g->n[1];
        } else {
            La.g0 = tab(HL.last_axis == 1 ? 0 : 1);
            La.g1 = nullptr;
            La.n1 = 1;
        }
        La.n_last = HL.n_last;
        rows = std::max(rows, HL.n_last);
    }
    A.sel = g->hist_sel;
    A.offsets = g->offsets;
    A.ds = (const DensStats *)g->dstats.p;
    A.ndim = nd;
    A.K = K;
    A.K_pad = K_pad;
    A.B = g->B;
    A.C = g->n_chunks;
    A.hist = hist;
    A.part = (float *)g->hist_part.p;
    A.dstatus = g->dstatus;
    const size_t smem = hist_smem_bytes(rows);
    // run-end words encode the rest index in 15 bits (3-D: a0 < 128, a1 < 256)
    const bool coded = nd == 2 || (g->n[0] <= 128 && g->n[1] <= 256);
    dim3 grd((unsigned)(A.C / kHistWarps), (unsigned)ceil_div64(K, kKT));
    {
        VUP_PROF("hist_segmented", s, 1);
        if (smem <= 220 * 1024 && coded) {
            if (nd == 3) {
                VUP_CHECK_CUDA(cudaFuncSetAttribute(k_hist_smem<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                k_hist_smem<2><<<grd, kHistWarps * 32, smem, s>>>(A, rows);
            } else {
                VUP_CHECK_CUDA(cudaFuncSetAttribute(k_hist_smem<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                k_hist_smem<1><<<grd, kHistWarps * 32, smem, s>>>(A, rows);
            }
        } else {
            k_hist_global<<<grd, kHistWarps * 32, 0, s>>>(A);
        }
        VUP_CHECK_LAUNCH();
    }
    VUP_PROF("hist_fixup", s, 1);
    dim3 fg((unsigned)ceil_div64(K, 128), (unsigned)g->B);
    k_hist_fixup<<<fg, 128, 0, s>>>(A);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}
