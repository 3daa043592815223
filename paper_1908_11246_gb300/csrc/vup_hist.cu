// Output probability vectors (Eq. 4 / Eq. 5, Eq. VUP): H[k, b] = sum of the
// normalised input probabilities of the grid points whose model value falls in
// bin b.  The one-hot model matrix of Eq. MUP is applied as a segmented
// reduction over the grid points pre-sorted by bin ("sort and sum").
//
// Layout: a warp serves 128 densities, four per lane; every lane walks the
// same sorted point stream, so control flow is uniform and one 16-byte gather
// per lane (128 consecutive shared-memory words per warp, conflict-free)
// yields four distribution-points.  Points are grouped in runs that share the sort key
// and every axis index but the gathered one: inside a run only the gathered
// axis' factor is read, from a shared-memory tile; the product with the other
// axes' factors is applied once per run.  Those factors are loaded four runs
// ahead: the run-end word of run r carries the rest index of run r + 4.  The
// point stream is staged into shared memory with bulk asynchronous copies
// (cp.async.bulk + mbarrier) and read four points per broadcast load.
//
// The gathered axis is cut into P parts so that one part's 64-density tile
// fits in shared memory; the stream is sorted by (part, bin) and every part
// is chunked separately.  Each warp owns a chunk; bins cut by chunk
// boundaries are written as partials, and a reduction kernel sums partials
// and parts in a fixed order (deterministic).  On 2-D grids two layouts exist
// (either axis gathered); the device uses the one with fewer runs.
#include "vup_internal.cuh"
#include "vup_async.cuh"

#include <algorithm>
#include <vector>

namespace {

constexpr int kHistWarps = 20;
constexpr int kChunksPerWarp = 4;                    // chunks per warp in the smallest group
constexpr int kGroupChunks = kHistWarps * kChunksPerWarp;  // chunks per part come in multiples of this
constexpr int kKT = 128;                     // densities per k-tile (four per lane)
constexpr int kWin = 128;                    // sorted-point words per staging buffer
constexpr int kMaxPartRows = 392;            // gathered-axis rows per shared-memory tile
constexpr int kRowShift = 9;                 // log2 of a tile row's bytes (kKT floats)
constexpr uint32_t kOffMask = 0x1ffu << kRowShift;  // row byte offset (rows < 512)
constexpr uint32_t kRunEnd = 1u << 30, kBinEnd = 1u << 31;
constexpr uint32_t kFlags = kRunEnd | kBinEnd;
constexpr uint32_t kSpin = 1u << 26;
constexpr int kPF = 16;                      // runs prefetched per block (global fallback)
constexpr int kRecBinsH = 8;                 // bins per record group (the layout builder's kRecBins)

struct LayoutArgs {
    const uint32_t *hpt;
    const int32_t *perm;   // sorted position -> flat index of the layout (global fallback)
    const int32_t *run_start, *run_rest, *run_bin;
    const int32_t *chunk_pt, *chunk_run, *chunk_bin;
    const int32_t *koff;   // key offsets [P * B + 1]
    const int2 *key_chunks;  // [P * B] first / last chunk of each key (-1 if empty)
    const uint2 *ipt;      // interval stream (word pairs)
    const int32_t *iv_rest, *chunk_iv;
    const uint4 *rec;      // record stream (two uint4 per record)
    const int32_t *rec_rest, *rec_goff;
    const int2 *rec_gch;   // first / last chunk holding each group
    const int32_t *rec_chunk, *rec_chunk_grp;
    const float *g_last;   // factor table of the gathered axis  [n_last][K_pad]
    const float *g0, *g1;  // rest-axis factor tables (g1 only for 3-D)
    int64_t n_last, part_rows;
    int64_t n1;            // size of the second rest axis (3-D)
    int64_t n0;            // rows of g0 (the first rest axis)
    int P;
};

struct HistArgs {
    LayoutArgs L0, L1;
    const int32_t *sel;   // device: chosen layout, stream (1 = intervals)
    const DensStats *ds;
    int ndim;
    int64_t K, K_pad;
    int B;
    int C;                // chunks per part
    int group_chunks;     // chunks per work item (a multiple of kGroupChunks dividing C)
    int rec_sets;         // record stream: work items per part (each a range of the part's record chunks)
    int C_rec;            // record chunks per part
    int GB;               // record groups per part: ceil(B / kRecBins)
    int points_only;      // 1: point stream whatever the layout choice says
    int rest_smem;        // 3-D point stream: both rest-axis factor tiles staged in shared memory
    int64_t rest_n0;      // rows of the first rest axis (3-D)
    float *hist;          // [K][B]
    float *part;          // [P * C][2][K_pad]
    float *direct;        // [P][K][B] (P > 1)
    const float *prefix;  // prefix-sum tiles [P][K_pad / 128][pre_rows][128] (null: each CTA sums its own)
    int64_t pre_rows;     // rows of a prefix tile (the most part rows + 1)
    int *dstatus;
};

__device__ __forceinline__ LayoutArgs pick(const HistArgs &A) { return A.sel[0] ? A.L1 : A.L0; }

using namespace vup_async;

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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

// Shared memory of k_hist_smem: the part's gathered-axis factor tile
// [rows + 1][64] (the extra row is zero; foreign points of a chunk's first
// and last group point at it), per warp 2 staging buffers of kWin point
// words, 2 mbarriers per warp.
__host__ __device__ inline size_t hist_tile_bytes(int64_t rows) { return (size_t)((rows + 1) * kKT * 4); }
__host__ __device__ inline size_t hist_warp_bytes() { return (size_t)2 * kWin * 4; }
// Kernel variants: 0 point stream, 1 interval stream, 2 record stream, 3
// record stream with 16 warps of up to 128 registers (more of its five
// gathers and four accumulators in flight per warp; measured faster when the
// rest-factor table stays in L2, slower when its rows come from HBM and more
// warps hide the latency), 4 point stream of a 3-D grid with both rest-axis
// factor tables staged in shared memory.  The others run 20 warps of 96
// registers.  Each fills the register file of the one CTA per SM that the
// tile allows.
__host__ __device__ constexpr int hist_warps(int mode) { return (mode == 2 || mode == 3) ? 16 : kHistWarps; }
__host__ __device__ constexpr int hist_stream_of(int mode) { return mode == 3 ? 2 : (mode == 4 ? 0 : mode); }
__host__ __device__ inline size_t hist_smem_bytes(int64_t rows, int warps = kHistWarps) {
    return hist_tile_bytes(rows) + warps * hist_warp_bytes() + warps * 2 * sizeof(uint64_t);
}

// Store the finished sums of key `key` for this lane's four densities (global
// fallback kernel: the normalisers are applied here).
struct Flusher {
    const HistArgs &A;
    const LayoutArgs &H;
    int c, p;
    int32_t p0, p1, first_key;
    int64_t k;
    float4 invZ;
    __device__ __forceinline__ void operator()(int32_t key, float4 v) const {
        const float4 val = make_float4(v.x * invZ.x, v.y * invZ.y, v.z * invZ.z, v.w * invZ.w);
        const bool shared = H.koff[key] < p0 || H.koff[key + 1] > p1;
        if (shared) {
            const int side = (key == first_key) ? 0 : 1;
            *reinterpret_cast<float4 *>(A.part + ((int64_t)c * 2 + side) * A.K_pad + k) = val;
        } else {
            *reinterpret_cast<float4 *>(A.direct + (int64_t)key * A.K_pad + k) = val;
        }
    }
};

__device__ __forceinline__ float inv_z(const HistArgs &A, int64_t k) {
    if (k >= A.K) return 0.f;
    double z = 1.0;
    for (int d = 0; d < A.ndim; ++d) z *= A.ds[k * A.ndim + d].invZ;
    return (float)z;
}

__device__ __forceinline__ float4 load_inv_z(const HistArgs &A, int64_t k) {
    return make_float4(inv_z(A, k), inv_z(A, k + 1), inv_z(A, k + 2), inv_z(A, k + 3));
}

// Four densities' values per lane, handled as two packed FP32 pairs: the
// .f32x2 forms round each half exactly as the scalar operation does, so the
// sums are bit-identical to four scalar FMAs / subtractions, in half the
// instructions.
__device__ __forceinline__ uint64_t pk2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 up2(uint64_t r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float4 from_pairs(uint64_t lo, uint64_t hi) {
    const float2 l = up2(lo), h = up2(hi);
    return make_float4(l.x, l.y, h.x, h.y);
}
__device__ __forceinline__ float4 ld4(const float *q) { return *reinterpret_cast<const float4 *>(q); }
__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
    uint64_t lo, hi;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(lo) : "l"(pk2(a.x, a.y)), "l"(pk2(b.x, b.y)));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(hi) : "l"(pk2(a.z, a.w)), "l"(pk2(b.z, b.w)));
    return from_pairs(lo, hi);
}
__device__ __forceinline__ float4 sub4(float4 a, float4 b) {
    uint64_t lo, hi;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(lo) : "l"(pk2(a.x, a.y)), "l"(pk2(b.x, b.y)));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(hi) : "l"(pk2(a.z, a.w)), "l"(pk2(b.z, b.w)));
    return from_pairs(lo, hi);
}
__device__ __forceinline__ void add4(float4 &a, float4 b) {
    uint64_t lo = pk2(a.x, a.y), hi = pk2(a.z, a.w);
    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(lo) : "l"(pk2(b.x, b.y)));
    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(hi) : "l"(pk2(b.z, b.w)));
    a = from_pairs(lo, hi);
}
__device__ __forceinline__ void fma4(float4 &a, float4 w, float4 b) {
    uint64_t lo = pk2(a.x, a.y), hi = pk2(a.z, a.w);
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(lo) : "l"(pk2(w.x, w.y)), "l"(pk2(b.x, b.y)));
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(hi) : "l"(pk2(w.z, w.w)), "l"(pk2(b.z, b.w)));
    a = from_pairs(lo, hi);
}

// Per-item context, kept in shared memory: the chosen layout, the output
// pointers and sizes.  Warps read it on demand, so none of it occupies
// registers across the point loop.
struct ItemCtx {
    LayoutArgs H;
    float *part;   // [P * C][2][K_pad] partial sums of keys cut by chunk bounds
    float *direct; // [P * B][K_pad] sums of keys held by one chunk
    int64_t K, K_pad;
    int B, C, group_chunks, rec_sets, C_rec, GB;
    int mode;      // 0: point stream, tile holds factors; 1: interval stream, tile holds prefix sums
    int rest_smem;  // (3-D point stream) rest-axis factors [n0][kKT], [n1][kKT] after the staging buffers
    int64_t rest_n0;
    const float *prefix;
    int64_t pre_rows;
    int *dstatus;
};

// Store the finished sums of one key for a lane's four densities (16 bytes,
// density-contiguous: one coalesced 512-byte row per warp): keys cut by the
// chunk bounds go to the chunk's partials (side 0 = its first key), the
// others to the key's row of the direct sums.  A one-part histogram also
// goes through the direct rows: scattered 4-byte stores into the [K][B]
// output from the point loop measured slower than the coalesced rows plus
// the finishing copy.  Out of line: it runs once per key, and keeping it
// out of the point loop keeps that loop's code small.
__device__ __noinline__ void flush_key(const ItemCtx *X, int c, int p, int64_t k, int32_t key, float4 v,
                                       bool shared, bool first) {
    float *dst = shared ? X->part + ((int64_t)c * 2 + (first ? 0 : 1)) * X->K_pad + k
                        : X->direct + (int64_t)key * X->K_pad + k;
    *reinterpret_cast<float4 *>(dst) = v;
}

// Interval stream of chunk c (part p): interval i adds f_i (P[b_i] - P[a_i])
// to its key's sum for the lane's four densities, P being the part's prefix
// sums in the shared-memory tile and f_i its rest-axis factor.  Every
// interval loads its own rest factor four intervals ahead into one of four
// registers (the interval's index mod 4), so the loop runs in steps of four
// intervals (two 16-byte broadcast loads of word pairs) and rotates nothing.
template <int NF>
__device__ __forceinline__ bool iv_chunk(const ItemCtx &X, int c, int p, int64_t k, const float *ws, uint32_t *win,
                                         uint64_t *mbar, uint32_t &wseq, volatile int *abort) {
    const LayoutArgs &H = X.H;
    const int lane = threadIdx.x & 31;
    const int32_t p0 = H.chunk_pt[c], p1 = H.chunk_pt[c + 1];
    if (p0 >= p1) return true;
    const int32_t i0 = H.chunk_iv[c], i1 = H.chunk_iv[c + 1];
    const int32_t r0 = H.chunk_run[c], r1 = H.chunk_run[c + 1];
    const int32_t first_key = H.chunk_bin[2 * c], last_key = H.chunk_bin[2 * c + 1];
    const bool sh_first = H.koff[first_key] < p0 || H.koff[first_key + 1] > p1;
    const bool sh_last = H.koff[last_key] < p0 || H.koff[last_key + 1] > p1;

    // words [w0, w1): intervals from i0 rounded down to a multiple of four
    const int32_t ib = i0 & ~3;
    const int32_t w0 = 2 * ib, w1 = 2 * i1;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(H.ipt);
    const int32_t wb0 = w0 & ~(kWin - 1);
    if (lane == 0) {
        const int b0 = wseq & 1;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of both buffers
        bulk_copy(win + b0 * kWin, src + wb0, kWin * 4, &mbar[b0]);
        if (wb0 + kWin < w1) bulk_copy(win + (b0 ^ 1) * kWin, src + wb0 + kWin, kWin * 4, &mbar[b0 ^ 1]);
    }
    __syncwarp();

    // rest-factor rows: this lane's four densities of row `row` (byte stride)
    const uint32_t stride = (uint32_t)(X.K_pad * 4);
    const char *g0b = reinterpret_cast<const char *>(H.g0 + k);
    const char *g1b = NF == 2 ? reinterpret_cast<const char *>(H.g1 + k) : nullptr;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto row4 = [&](const char *base, uint32_t row) -> float4 {
        return *reinterpret_cast<const float4 *>(base + (uint64_t)row * stride);
    };
    // factor of interval i + 4 from interval i's code: 9 low bits below the row
    // field and 12 bits above it (2-D: the rest index; 3-D: a0 low, a1 high)
    // (debug build: rows outside the factor tables are recorded and read as row 0)
    auto rest2 = [&](uint32_t a0, uint32_t a1) -> float4 {
        if (!VUP_DBG_IN(a0, H.n0, X.dstatus)) a0 = 0;
        if (!VUP_DBG_IN(a1, H.n1, X.dstatus)) a1 = 0;
        return mul4(row4(g0b, a0), row4(g1b, a1));
    };
    auto rest1 = [&](uint32_t a0) -> float4 {
        if (!VUP_DBG_IN(a0, H.n0, X.dstatus)) a0 = 0;
        return row4(g0b, a0);
    };
    auto coded_factor = [&](uint32_t u) -> float4 {
        if (NF == 2) return rest2(u & 0x1ffu, (u >> 18) & 0xfffu);
        return rest1((u & 0x1ffu) | ((u >> 9) & (0xfffu << 9)));
    };
    auto first_factor = [&](int32_t i) -> float4 {
        if (i < i0 || i >= i1) return zero4;
        const int32_t rest = H.iv_rest[i];
        if (NF == 2) {
            const int32_t a0 = rest / (int32_t)H.n1;
            return rest2((uint32_t)a0, (uint32_t)(rest - a0 * (int32_t)H.n1));
        }
        return rest1((uint32_t)rest);
    };
    float4 f0 = first_factor(ib), f1 = first_factor(ib + 1), f2 = first_factor(ib + 2), f3 = first_factor(ib + 3);

    float4 bacc = zero4;
    int32_t r = r0, cur_key = first_key;
    const uint32_t wsl = smem_u32(ws) + lane * 16;
    auto gather = [&](uint32_t addr) -> float4 {
        float4 v;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "r"(addr));
        return v;
    };
    auto flush = [&](int32_t key, float4 v) {
        const bool first = key == first_key;
        flush_key(&X, c, p, k, key, v, first ? sh_first : (key == last_key && sh_last), first);
    };
    auto step = [&](uint32_t x, uint32_t y, float4 &f) {
        uint32_t xo = x, yo = y & kOffMask;  // (debug build: rows past the tile are recorded, read as row 0)
        if (!VUP_DBG_IN(xo >> kRowShift, X.pre_rows, X.dstatus)) xo = 0;
        if (!VUP_DBG_IN(yo >> kRowShift, X.pre_rows, X.dstatus)) yo = 0;
        const float4 pa = gather(wsl + xo), pb = gather(wsl + yo);
        fma4(bacc, f, sub4(pb, pa));
        f = coded_factor(y);
        if (y & kBinEnd) {
            if (VUP_DBG_IN(cur_key, (int64_t)H.P * X.B, X.dstatus)) flush(cur_key, bacc);
            bacc = zero4;
            cur_key = r + 1 < r1 ? H.run_bin[r + 1] : -1;
        }
        r += (y >> 30) & 1u;  // run end
    };
    // foreign intervals read row 0 twice (difference 0) and carry no flags;
    // those before the chunk keep their rest codes (they load the chunk's first factors)
    constexpr uint32_t kCodes = ~(kOffMask | kFlags);
    auto masked = [&](uint32_t &x, uint32_t &y, int32_t i) {
        if (i < i0) {
            x = 0u;
            y &= kCodes;
        } else if (i >= i1) {
            x = 0u;
            y = 0u;
        }
    };

    for (int32_t wbase = wb0; wbase < w1; wbase += kWin, ++wseq) {
        const int b = wseq & 1;
        for (uint32_t i = 0; !mbar_try_wait(&mbar[b], (wseq >> 1) & 1); ++i) {
            if (i > kSpin || *abort) {  // a staged copy never landed: record and stop
                *abort = 1;
                atomicCAS(X.dstatus, 0, VUP_DSTAT_TIMEOUT);
                return false;
            }
        }
        const uint32_t *wv = win + b * kWin;
        const int lo = (w0 > wbase ? w0 : wbase) - wbase;
        const int hi = (w1 < wbase + kWin ? w1 : wbase + kWin) - wbase;
        for (int q = lo; q < hi; q += 8) {
            uint4 u0 = *reinterpret_cast<const uint4 *>(wv + q), u1 = *reinterpret_cast<const uint4 *>(wv + q + 4);
            const int32_t iq = (wbase + q) >> 1;
            if (iq < i0 || iq + 4 > i1) {
                masked(u0.x, u0.y, iq);
                masked(u0.z, u0.w, iq + 1);
                masked(u1.x, u1.y, iq + 2);
                masked(u1.z, u1.w, iq + 3);
            }
            step(u0.x, u0.y, f0);
            step(u0.z, u0.w, f1);
            step(u1.x, u1.y, f2);
            step(u1.z, u1.w, f3);
        }
        __syncwarp();
        if (lane == 0 && wbase + 2 * kWin < w1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bulk_copy(win + b * kWin, src + wbase + 2 * kWin, kWin * 4, &mbar[b]);
        }
    }
    if (cur_key >= 0) flush(cur_key, bacc);
    return true;
}

// Record stream, chunk c of part p: record t adds s_t f_t (P[B_j+1] - P[B_j])
// to bin 8q + j, j = 0..7: a gather of P[B_0] and four more for each half of
// the group that holds a bin, one rest-factor load four records ahead, s_t
// its sign; a group's eight sums are stored when its last record passes (groups
// cut by the chunk bounds -- only its first and last -- go to the chunk's
// partial rows, as keys do on the other streams).
constexpr uint32_t kRecNegFlag = 1u << 30;
constexpr uint32_t kRecEndFlag = 1u << 31;

// Store a record group's eight sums (a lane's four densities each): whole
// groups to their direct rows, cut ones to the chunk's partial rows (side 0:
// its first group).  Out of line, like flush_key: it runs once per group.
__device__ __noinline__ void flush_group(const ItemCtx *X, int c, int p, int64_t k, int32_t gr, bool shared,
                                         bool first, float4 a0, float4 a1, float4 a2, float4 a3, float4 a4,
                                         float4 a5, float4 a6, float4 a7) {
    const int b0 = (gr - p * X->GB) * kRecBinsH;
    const int64_t K_pad = X->K_pad;
    float *row = shared ? X->part + ((int64_t)c * 2 + (first ? 0 : 1)) * kRecBinsH * K_pad + k
                        : X->direct + ((int64_t)p * X->B + b0) * K_pad + k;
    const float4 a[kRecBinsH] = {a0, a1, a2, a3, a4, a5, a6, a7};
#pragma unroll
    for (int j = 0; j < kRecBinsH; ++j)
        if (shared || b0 + j < X->B) *reinterpret_cast<float4 *>(row + j * K_pad) = a[j];
}
template <int NF>
__device__ __forceinline__ bool rec_chunk_walk(const ItemCtx &X, int c, int p, int64_t k, const float *ws,
                                               uint32_t *win, uint64_t *mbar, uint32_t &wseq, volatile int *abort) {
    const LayoutArgs &H = X.H;
    const int lane = threadIdx.x & 31;
    const int32_t r0 = H.rec_chunk[c], r1 = H.rec_chunk[c + 1];
    if (r0 >= r1) return true;
    const int32_t first_grp = H.rec_chunk_grp[2 * c], last_grp = H.rec_chunk_grp[2 * c + 1];
    // a group is cut when it starts before or ends after the chunk
    const bool sh_first = H.rec_goff[first_grp] < r0 || H.rec_goff[first_grp + 1] > r1;
    const bool sh_last = H.rec_goff[last_grp] < r0 || H.rec_goff[last_grp + 1] > r1;
    const bool last_ends = (H.rec[2 * (int64_t)(r1 - 1) + 1].x & kRecEndFlag) != 0;
    // words [w0, w1): records from r0 rounded down to a multiple of four
    const int32_t rb = r0 & ~3;
    const int64_t w0 = 8 * (int64_t)rb, w1 = 8 * (int64_t)r1;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(H.rec);
    const int64_t wb0 = w0 & ~(int64_t)(kWin - 1);
    if (lane == 0) {
        const int b0 = wseq & 1;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of both buffers
        bulk_copy(win + b0 * kWin, src + wb0, kWin * 4, &mbar[b0]);
        if (wb0 + kWin < w1) bulk_copy(win + (b0 ^ 1) * kWin, src + wb0 + kWin, kWin * 4, &mbar[b0 ^ 1]);
    }
    __syncwarp();

    const uint32_t stride = (uint32_t)(X.K_pad * 4);
    const char *g0b = reinterpret_cast<const char *>(H.g0 + k);
    const char *g1b = NF == 2 ? reinterpret_cast<const char *>(H.g1 + k) : nullptr;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto row4 = [&](const char *base, uint32_t row) -> float4 {
        return *reinterpret_cast<const float4 *>(base + (uint64_t)row * stride);
    };
    // rest factor from a record's code (2-D: the rest index; 3-D: a0 | a1 << 15)
    // (debug build: rows outside the factor tables are recorded and read as row 0)
    auto rest2 = [&](uint32_t a0, uint32_t a1) -> float4 {
        if (!VUP_DBG_IN(a0, H.n0, X.dstatus)) a0 = 0;
        if (!VUP_DBG_IN(a1, H.n1, X.dstatus)) a1 = 0;
        return mul4(row4(g0b, a0), row4(g1b, a1));
    };
    auto rest1 = [&](uint32_t a0) -> float4 {
        if (!VUP_DBG_IN(a0, H.n0, X.dstatus)) a0 = 0;
        return row4(g0b, a0);
    };
    auto coded_factor = [&](uint32_t u) -> float4 {
        if (NF == 2) return rest2(u & 0x7fffu, u >> 15);
        return rest1(u);
    };
    auto first_factor = [&](int32_t t) -> float4 {
        if (t < r0 || t >= r1) return zero4;
        const int32_t rest = H.rec_rest[t];
        if (NF == 2) {
            const int32_t a0 = rest / (int32_t)H.n1;
            return rest2((uint32_t)a0, (uint32_t)(rest - a0 * (int32_t)H.n1));
        }
        return rest1((uint32_t)rest);
    };
    float4 f0 = first_factor(rb), f1 = first_factor(rb + 1), f2 = first_factor(rb + 2), f3 = first_factor(rb + 3);

    float4 acc[kRecBinsH];
#pragma unroll
    for (int j = 0; j < kRecBinsH; ++j) acc[j] = zero4;
    // a group's eight sums: whole groups to their direct rows, cut ones to the chunk's partials
    auto flush = [&](int32_t gr) {
        const bool first = gr == first_grp;
        if (VUP_DBG_IN(gr - p * X.GB, X.GB, X.dstatus))  // (debug build: a group outside the part is skipped)
            flush_group(&X, c, p, k, gr, first ? sh_first : (gr == last_grp && sh_last), first, acc[0], acc[1], acc[2],
                    acc[3], acc[4], acc[5], acc[6], acc[7]);
#pragma unroll
        for (int j = 0; j < kRecBinsH; ++j) acc[j] = zero4;
    };
    const uint32_t wsl = smem_u32(ws) + lane * 16;
    auto gather = [&](uint32_t addr) -> float4 {
        float4 v;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "r"(addr));
        return v;
    };
    auto step = [&](const uint4 u, const uint4 v, float4 &f) {
        // boundary rows B_0..B_8 (16 bits each); bins with B_j+1 == B_j are absent
        uint32_t rw[kRecBinsH + 1] = {u.x & 0xffffu, u.x >> 16, u.y & 0xffffu, u.y >> 16, u.z & 0xffffu,
                                      u.z >> 16,     u.w & 0xffffu, u.w >> 16, v.x & 0xffffu};
#ifdef VUP_DEBUG
        // (debug build: a boundary row past the tile makes the record empty)
        bool rows_ok = true;
#pragma unroll
        for (int j = 0; j <= kRecBinsH; ++j) rows_ok = rows_ok && VUP_DBG_IN(rw[j], X.pre_rows, X.dstatus);
        if (!rows_ok)
#pragma unroll
            for (int j = 0; j <= kRecBinsH; ++j) rw[j] = 0;
#endif
        const float4 fs = (v.x & kRecNegFlag) ? make_float4(-f.x, -f.y, -f.z, -f.w) : f;
        // each half of the group is skipped when it holds no bin (its
        // boundaries then all equal its first)
        float4 prev = gather(wsl + (rw[0] << kRowShift));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            constexpr int kH = kRecBinsH / 2;
            if (rw[kH * h + kH] != rw[kH * h]) {
#pragma unroll
                for (int j = kH * h; j < kH * h + kH; ++j) {
                    const float4 nx = gather(wsl + (rw[j + 1] << kRowShift));
                    fma4(acc[j], fs, sub4(nx, prev));
                    prev = nx;
                }
            }
        }
        f = coded_factor(v.y);
        if (__builtin_expect((v.x & kRecEndFlag) != 0, 0)) flush((int32_t)v.z);
    };
    // foreign records: every boundary row 0 (differences 0), no group end;
    // those before the chunk keep their rest codes (they load its first factors)
    auto masked = [&](uint4 &u, uint4 &v, int32_t t) {
        if (t < r0) {
            u = make_uint4(0u, 0u, 0u, 0u);
            v = make_uint4(0u, v.y, 0u, 0u);
        } else if (t >= r1) {
            u = make_uint4(0u, 0u, 0u, 0u);
            v = make_uint4(0u, 0u, 0u, 0u);
        }
    };

    for (int64_t wbase = wb0; wbase < w1; wbase += kWin, ++wseq) {
        const int b = wseq & 1;
        for (uint32_t i = 0; !mbar_try_wait(&mbar[b], (wseq >> 1) & 1); ++i) {
            if (i > kSpin || *abort) {  // a staged copy never landed: record and stop
                *abort = 1;
                atomicCAS(X.dstatus, 0, VUP_DSTAT_TIMEOUT);
                return false;
            }
        }
        const uint4 *wq = reinterpret_cast<const uint4 *>(win + b * kWin);
        const int lo = (int)((w0 > wbase ? w0 : wbase) - wbase);
        const int hi = (int)((w1 < wbase + kWin ? w1 : wbase + kWin) - wbase);
        for (int qq = lo; qq < hi; qq += 32) {
            const int32_t t0 = (int32_t)((wbase + qq) >> 3);
            const bool edge = t0 < r0 || t0 + 4 > r1;
            auto one = [&](int m, float4 &f) {
                uint4 u = wq[qq / 4 + 2 * m], v = wq[qq / 4 + 2 * m + 1];
                if (__builtin_expect(edge, 0)) masked(u, v, t0 + m);
                step(u, v, f);
            };
            one(0, f0);
            one(1, f1);
            one(2, f2);
            one(3, f3);
        }
        __syncwarp();
        if (lane == 0 && wbase + 2 * kWin < w1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bulk_copy(win + b * kWin, src + wbase + 2 * kWin, kWin * 4, &mbar[b]);
        }
    }
    if (!last_ends) flush(last_grp);  // the chunk ends inside its last group
    return true;
}

// One work item: part p, chunk group cg (kGroupChunks chunks, drawn by the
// warps one at a time) and
// the 128 densities from k0 of the instance *Ap (kernel parameter or global
// memory).  Called by every thread of the CTA; `wseq` counts the staging
// windows this warp has consumed so far (it keeps the per-warp mbarrier
// phases consistent across items).
template <int NF, int MODE>
__device__ __forceinline__ void hist_item(const HistArgs *Ap, int p, int cg, int64_t k0, uint8_t *sm,
                                          int64_t tile_rows, uint32_t &wseq, volatile int *abort, ItemCtx &X,
                                          float *s_invz, int *next_chunk) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k = k0 + 4 * lane;
    float *ws = reinterpret_cast<float *>(sm);
    const size_t tb = hist_tile_bytes(tile_rows);
    uint32_t *win = reinterpret_cast<uint32_t *>(sm + tb + (size_t)warp * hist_warp_bytes());
    constexpr int kWarps = hist_warps(MODE);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + tb + kWarps * hist_warp_bytes()) + 2 * warp;

    // the previous item's readers of the tile and the context are done first
    __syncthreads();
    if (*abort) return;  // a wait of an earlier item expired (uniform: read after the barrier)
    if (threadIdx.x == 0) {
        const HistArgs &A = *Ap;
        *next_chunk = 0;
        X.H = A.sel[0] ? A.L1 : A.L0;
        X.part = A.part;
        X.direct = A.direct;
        X.K = A.K;
        X.K_pad = A.K_pad;
        X.B = A.B;
        X.C = A.C;
        X.group_chunks = A.group_chunks;
        X.rec_sets = A.rec_sets;
        X.C_rec = A.C_rec;
        X.GB = A.GB;
        X.mode = hist_stream_of(MODE);
        X.prefix = A.prefix;
        X.pre_rows = A.pre_rows;
        X.dstatus = A.dstatus;
        X.rest_smem = MODE == 4 ? 1 : 0;
        X.rest_n0 = A.rest_n0;
    }
    if (threadIdx.x < kKT) s_invz[threadIdx.x] = inv_z(*Ap, k0 + threadIdx.x);
    __syncthreads();
    const LayoutArgs &H = X.H;
    if (p >= H.P) return;  // uniform
    // this part's rows of the gathered-axis factor table (16-byte asynchronous
    // copies) + a zero row, then every column scaled by its density's
    // normaliser 1 / prod_d Z_d
    const int64_t row0 = (int64_t)p * H.part_rows;
    const int64_t nrows = min(H.part_rows, H.n_last - row0);
    constexpr bool kPrefixTile = hist_stream_of(MODE) != 0;  // interval / record streams: prefix sums
    const bool pre = kPrefixTile && X.prefix != nullptr;     // the prefix sums come ready-made
    if (pre) {
        const float *src = X.prefix + ((int64_t)p * (X.K_pad / kKT) + k0 / kKT) * X.pre_rows * kKT;
        for (int64_t e = threadIdx.x; e < (nrows + 1) * (kKT / 4); e += blockDim.x) cp_async16(ws + e * 4, src + e * 4);
    } else {
        const float *src = H.g_last + row0 * X.K_pad + k0;
        const int64_t K_pad = X.K_pad;
        for (int64_t e = threadIdx.x; e < nrows * (kKT / 4); e += blockDim.x) {
            const int64_t a = e / (kKT / 4), cc = e % (kKT / 4);
            cp_async16(ws + a * kKT + cc * 4, src + a * K_pad + cc * 4);
        }
    }
    if (MODE == 4) {
        // the k-tile's rows of both rest-axis factor tables (unnormalised)
        float *rs = reinterpret_cast<float *>(sm + hist_smem_bytes(tile_rows, kWarps));
        const int64_t n0 = X.rest_n0, n1 = H.n1, K_pad = X.K_pad;
        for (int64_t e = threadIdx.x; e < (n0 + n1) * (kKT / 4); e += blockDim.x) {
            const int64_t a = e / (kKT / 4), cc = e % (kKT / 4);
            const float *src = a < n0 ? H.g0 + a * K_pad : H.g1 + (a - n0) * K_pad;
            cp_async16(rs + a * kKT + cc * 4, src + k0 + cc * 4);
        }
    }
    cp_async_commit();
    if (!pre && threadIdx.x < kKT) ws[nrows * kKT + threadIdx.x] = 0.f;
    cp_async_wait_all();
    __syncthreads();
    if (pre) {
        // the staging buffers are next written by bulk copies (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    } else if (kPrefixTile) {
        // interval stream: every column becomes the exclusive prefix sums
        // P[0..nrows] of its scaled factors (compensated sums, each P rounded
        // once to FP32), so that rows a .. b - 1 sum to P[b] - P[a].  The
        // rows are cut into kScanSegs segments, one thread per (segment,
        // column): segment totals first (kept in the idle staging buffers),
        // then each segment rescanned from the sum of the totals before it.
        constexpr int kScanSegs = kWarps * 32 / kKT;
        const int col = threadIdx.x % kKT, sg = threadIdx.x / kKT;
        const int64_t rs = (nrows + kScanSegs - 1) / kScanSegs;
        const int64_t a0 = min(nrows, sg * rs), a1 = min(nrows, a0 + rs);
        const float iz = s_invz[col];
        float *tcol = ws + col;
        float2 *segsum = reinterpret_cast<float2 *>(sm + tb);  // [kScanSegs][kKT]
        auto add = [](float &sh, float &sl, float v) {
            const float t = sh + v, bb = t - sh;
            sl += (sh - (t - bb)) + (v - bb);
            sh = t;
        };
        {
            float sh = 0.f, sl = 0.f;
            for (int64_t a = a0; a < a1; ++a) add(sh, sl, tcol[a * kKT] * iz);
            segsum[sg * kKT + col] = make_float2(sh, sl);
        }
        __syncthreads();
        float oh = 0.f, ol = 0.f;
        for (int q = 0; q < sg; ++q) {
            const float2 v = segsum[q * kKT + col];
            add(oh, ol, v.x);
            ol += v.y;
        }
        for (int64_t a = a0; a < a1; ++a) {
            const float v = tcol[a * kKT] * iz;
            tcol[a * kKT] = oh + ol;
            add(oh, ol, v);
        }
        if (a1 == nrows && (a0 < a1 || sg == 0)) tcol[nrows * kKT] = oh + ol;
        // the staging buffers are next written by bulk copies (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    } else {
        for (int64_t e = threadIdx.x; e < nrows * kKT; e += blockDim.x) ws[e] *= s_invz[e % kKT];
    }
    __syncthreads();

    // the item's chunks are handed out one at a time (at least kChunksPerWarp per warp
    // on average), so a warp that drew short chunks takes another instead of
    // idling at the next item's barrier
    auto run_chunk = [&](const int wc) -> bool {
        const int c = p * X.C + wc;
        const int32_t p0 = H.chunk_pt[c], p1 = H.chunk_pt[c + 1];
        if (p0 >= p1) return true;
        const int32_t r0 = H.chunk_run[c], r1 = H.chunk_run[c + 1];
        // keys cut by the chunk bounds can only be its first and last key
        const int32_t first_key = H.chunk_bin[2 * c], last_key = H.chunk_bin[2 * c + 1];
        const bool sh_first = H.koff[first_key] < p0 || H.koff[first_key + 1] > p1;
        const bool sh_last = H.koff[last_key] < p0 || H.koff[last_key + 1] > p1;
        auto flush = [&](int32_t key, float4 v) {
            const bool first = key == first_key;
            flush_key(&X, c, p, k, key, v, first ? sh_first : (key == last_key && sh_last), first);
        };

        // staging of the sorted point stream: window i of this item lands in
        // buffer (wseq + i) & 1
        const uint32_t *hpt = H.hpt;
        const int32_t wb0 = p0 & ~(kWin - 1);
        if (lane == 0) {
            const int b0 = wseq & 1;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier items' reads of both buffers
            bulk_copy(win + b0 * kWin, hpt + wb0, kWin * 4, &mbar[b0]);
            if (wb0 + kWin < p1) bulk_copy(win + (b0 ^ 1) * kWin, hpt + wb0 + kWin, kWin * 4, &mbar[b0 ^ 1]);
        }
        __syncwarp();

        // rest-axis factors (four densities) of runs r .. r + 3, rotated through registers
        const int64_t K_pad = X.K_pad;
        const float *g0k = H.g0 + k;
        const float *g1k = NF == 2 ? H.g1 + k : nullptr;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        // 3-D: the product of the two rest axes' rows; with the rows staged in
        // shared memory (MODE 4) the first axis' row is kept in registers while
        // consecutive runs share it (95% of them on the 3-D workload: runs of
        // a bin are ordered by line)
        constexpr bool rs = NF == 2 && MODE == 4;
        const float *w0s = reinterpret_cast<const float *>(sm + hist_smem_bytes(tile_rows, kWarps)) + 4 * lane;
        const float *w1s = w0s + X.rest_n0 * kKT;
        uint32_t a0c = 0xffffffffu;
        float4 w0c = zero4;
        auto rest_rows = [&](uint32_t a0, uint32_t a1) -> float4 {
            // (debug build: rows outside the factor tables are recorded and read as row 0)
            if (!VUP_DBG_IN(a0, H.n0, X.dstatus)) a0 = 0;
            if (!VUP_DBG_IN(a1, H.n1, X.dstatus)) a1 = 0;
            if (rs) {
                if (a0 != a0c) {  // uniform: every lane follows the same run
                    w0c = ld4(w0s + a0 * kKT);
                    a0c = a0;
                }
                return mul4(w0c, ld4(w1s + a1 * kKT));
            }
            return mul4(ld4(g0k + (int64_t)a0 * K_pad), ld4(g1k + (int64_t)a1 * K_pad));
        };
        auto rest_factor = [&](int32_t r) -> float4 {
            if (r >= r1) return zero4;
            const int32_t rest = H.run_rest[r];
            if (NF == 2) {
                const int32_t a0 = rest / (int32_t)H.n1, a1 = rest - a0 * (int32_t)H.n1;
                return rest_rows((uint32_t)a0, (uint32_t)a1);
            }
            return ld4(g0k + (VUP_DBG_IN(rest, H.n0, X.dstatus) ? rest : 0) * K_pad);
        };
        // fc = factor of the current run, f1..f3 those of the next three runs
        // (MODE 4: shared-memory factors, no look-ahead: fc only)
        float4 fc = rest_factor(r0), f1 = zero4, f2 = zero4, f3 = zero4;
        if (!rs) {
            f1 = rest_factor(r0 + 1);
            f2 = rest_factor(r0 + 2);
            f3 = rest_factor(r0 + 3);
        }
        // factor of run r + 4 (MODE 4: r + 1), decoded from run r's end word: 9
        // low bits below the row field and 12 bits above it
        auto coded_factor = [&](uint32_t u) -> float4 {
            if (NF == 2) return rest_rows(u & 0x1ffu, (u >> 18) & 0xfffu);
            const uint32_t idx = (u & 0x1ffu) | (((u >> 18) & 0xfffu) << 9);
            return ld4(g0k + (int64_t)(VUP_DBG_IN(idx, H.n0, X.dstatus) ? idx : 0u) * K_pad);
        };

        // every point's factor is multiplied by its run's rest-axis factor fc as it
        // is added (one FMA per density, the same count as a plain add), so a run
        // end only advances the factor pipeline
        int32_t r = r0, cur_key = first_key;
        float4 bacc = zero4;
        const uint32_t wsl = smem_u32(ws) + lane * 16;
        const uint32_t null_word = (uint32_t)nrows << kRowShift;  // zero row, no flags

        auto run_end = [&](uint32_t u) {
            if (u & kBinEnd) {
                if (VUP_DBG_IN(cur_key, (int64_t)H.P * X.B, X.dstatus)) flush(cur_key, bacc);
                bacc = zero4;
                cur_key = r + 1 < r1 ? H.run_bin[r + 1] : -1;
            }
            if (rs) {
                fc = r + 1 < r1 ? coded_factor(u) : zero4;
            } else {
                fc = f1;
                f1 = f2;
                f2 = f3;
                f3 = coded_factor(u);
            }
            ++r;
        };
        auto gather = [&](uint32_t addr) -> float4 {
            float4 v;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                         : "r"(addr));
            return v;
        };
        // words without flags carry nothing but the row byte offset (run codes sit
        // on run-end words only), so the common path needs no masking
#ifdef VUP_DEBUG
        // (debug build: a row offset past the tile is recorded and read as the zero row 0)
        auto dbg_word = [&](uint32_t w) -> uint32_t {
            if ((w & kFlags) == 0)
                return VUP_DBG_IN(w >> kRowShift, nrows + 1, X.dstatus) && (w & ~kOffMask) == 0 ? w : 0u;
            return VUP_DBG_IN((w & kOffMask) >> kRowShift, nrows + 1, X.dstatus) ? w : (w & ~kOffMask);
        };
#endif
        auto group = [&](uint4 v) {
#ifdef VUP_DEBUG
            v = make_uint4(dbg_word(v.x), dbg_word(v.y), dbg_word(v.z), dbg_word(v.w));
#endif
            if (((v.x | v.y | v.z | v.w) & kFlags) == 0) {
                const float4 a0 = gather(wsl + v.x), a1 = gather(wsl + v.y), a2 = gather(wsl + v.z),
                             a3 = gather(wsl + v.w);
                fma4(bacc, fc, a0);
                fma4(bacc, fc, a1);
                fma4(bacc, fc, a2);
                fma4(bacc, fc, a3);
            } else {
                const float4 a0 = gather(wsl + (v.x & kOffMask)), a1 = gather(wsl + (v.y & kOffMask)),
                             a2 = gather(wsl + (v.z & kOffMask)), a3 = gather(wsl + (v.w & kOffMask));
                fma4(bacc, fc, a0);
                if (v.x & kFlags) run_end(v.x);
                fma4(bacc, fc, a1);
                if (v.y & kFlags) run_end(v.y);
                fma4(bacc, fc, a2);
                if (v.z & kFlags) run_end(v.z);
                fma4(bacc, fc, a3);
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

        for (int32_t wbase = wb0; wbase < p1; wbase += kWin, ++wseq) {
            const int b = wseq & 1;
            for (uint32_t i = 0; !mbar_try_wait(&mbar[b], (wseq >> 1) & 1); ++i) {
                if (i > kSpin || *abort) {  // a staged copy never landed: record and stop
                    *abort = 1;
                    atomicCAS(X.dstatus, 0, VUP_DSTAT_TIMEOUT);
                    return false;
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
                bulk_copy(win + b * kWin, hpt + wbase + 2 * kWin, kWin * 4, &mbar[b]);
            }
        }
        if (cur_key >= 0) flush(cur_key, bacc);
        return true;
    };
    if constexpr (hist_stream_of(MODE) == 2) {
        // this item's range of the part's record chunks, handed out one at a time
        const int c_lo = (int)((int64_t)cg * X.C_rec / X.rec_sets), c_hi = (int)((int64_t)(cg + 1) * X.C_rec / X.rec_sets);
        for (;;) {
            int ci = 0;
            if (lane == 0) ci = atomicAdd(next_chunk, 1);
            ci = __shfl_sync(0xffffffffu, ci, 0);
            if (c_lo + ci >= c_hi) break;
            if (!rec_chunk_walk<NF>(X, p * X.C_rec + c_lo + ci, p, k, ws, win, mbar, wseq, abort)) return;
        }
    } else {
        for (;;) {
            int ci = 0;
            if (lane == 0) ci = atomicAdd(next_chunk, 1);
            ci = __shfl_sync(0xffffffffu, ci, 0);
            if (ci >= X.group_chunks) break;
            const int wc = cg * X.group_chunks + ci;
            bool ok;
            if constexpr (MODE == 1) ok = iv_chunk<NF>(X, p * X.C + wc, p, k, ws, win, mbar, wseq, abort);
            else ok = run_chunk(wc);
            if (!ok) return;
        }
    }
}

__device__ __forceinline__ uint64_t *hist_mbar(uint8_t *sm, int64_t tile_rows, int warps) {
    return reinterpret_cast<uint64_t *>(sm + hist_tile_bytes(tile_rows) + warps * hist_warp_bytes()) +
           2 * (threadIdx.x >> 5);
}
__device__ __forceinline__ void hist_init_mbar(uint8_t *sm, int64_t tile_rows, int warps) {
    if ((threadIdx.x & 31) == 0) {
        uint64_t *mbar = hist_mbar(sm, tile_rows, warps);
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
}

// Stream of an instance's histogram: 1 = intervals (the layout's choice,
// unless the caller asked for points).
__device__ __forceinline__ int hist_stream(const HistArgs &A) { return A.points_only ? 0 : A.sel[1]; }

// One CTA per item, it = (k-tile * P + part) * G + chunk group, so that
// CTAs running together share k-tiles (rest-factor rows stay in L2) and the
// hardware hands items to SMs as they free up (item costs vary; a static
// split of items over persistent CTAs measured 12 % slower on the 3-D
// workload).  Each stream is its own kernel (their register allocations
// stay apart); the host launches both and every CTA of the one the device
// did not choose returns at once.
template <int NF, int MODE>
__global__ void __launch_bounds__(hist_warps(MODE) * 32, 1)
    k_hist_smem(const __grid_constant__ HistArgs A, int64_t tile_rows, int P, int G, int n_items) {
    pdl_trigger();
    pdl_wait();
    if (hist_stream(A) != hist_stream_of(MODE)) return;  // uniform
    extern __shared__ __align__(128) uint8_t sm[];
    __shared__ ItemCtx X;
    __shared__ float s_invz[kKT];
    __shared__ int abort, next_chunk;
    if (threadIdx.x == 0) abort = 0;
    hist_init_mbar(sm, tile_rows, hist_warps(MODE));
    uint32_t wseq = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int cg = it % G, pk = it / G;
        const int p = pk % P, kt = pk / P;
        hist_item<NF, MODE>(&A, p, cg, (int64_t)kt * kKT, sm, tile_rows, wseq, &abort, X, s_invz, &next_chunk);
    }
}

// Batched form: one persistent launch per stream over the work items of
// many instances (each with its own grid, densities and outputs), longest
// items first; items of instances on the other stream are skipped.
struct HistItem {
    int32_t inst, p, cg, kt;
};

// Per-stream item lists of a batch: the items of the instances whose
// device-chosen stream s is served by launch s, in the plan's (longest
// first) order, so that no launch walks past the other streams' items.  One
// CTA: the instances' streams to shared memory (global reads past
// kSplitStaged instances), then the items in blocks of kSplitThreads, each
// block compacted in order by warp ballots and per-warp counts.
constexpr int kSplitThreads = 1024;
constexpr int kSplitStaged = 32768;
__global__ void __launch_bounds__(kSplitThreads) k_hist_split_items(const HistArgs *__restrict__ insts, int n_inst,
                                                                    const HistItem *__restrict__ items, int n_items,
                                                                    int32_t *__restrict__ lists,
                                                                    int32_t *__restrict__ counts) {
    extern __shared__ uint8_t s_stream[];  // [n_inst] when staged
    __shared__ int s_warp[3][kSplitThreads / 32];
    __shared__ int s_base[3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool staged = n_inst <= kSplitStaged;
    if (staged)
        for (int i = tid; i < n_inst; i += blockDim.x) s_stream[i] = (uint8_t)min(hist_stream(insts[i]), 3);
    if (tid < 3) s_base[tid] = 0;
    __syncthreads();
    for (int base = 0; base < n_items; base += kSplitThreads) {
        const int it = base + tid;
        int st = 3;  // 3: no launch serves it
        if (it < n_items) {
            const int inst = items[it].inst;
            st = staged ? (int)s_stream[inst] : min(hist_stream(insts[inst]), 3);
        }
        unsigned m[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) m[q] = __ballot_sync(0xffffffffu, st == q);
        if (lane < 3) s_warp[lane][warp] = __popc(m[lane]);
        __syncthreads();
        if (st < 3) {
            int off = s_base[st] + __popc(m[st] & ((1u << lane) - 1u));
            for (int w = 0; w < warp; ++w) off += s_warp[st][w];
            lists[(int64_t)st * n_items + off] = it;
        }
        __syncthreads();
        if (tid < 3) {
            int t = 0;
            for (int w = 0; w < kSplitThreads / 32; ++w) t += s_warp[tid][w];
            s_base[tid] += t;
        }
        __syncthreads();
    }
    if (tid < 3) counts[tid] = s_base[tid];
}

template <int NF, int MODE>
__global__ void __launch_bounds__(hist_warps(MODE) * 32, 1) k_hist_batched(const HistArgs *__restrict__ insts,
                                                                     const HistItem *__restrict__ items,
                                                                     const int32_t *__restrict__ list,
                                                                     const int32_t *__restrict__ count,
                                                                     int64_t tile_rows,
                                                                     int *__restrict__ next_item) {
    extern __shared__ __align__(128) uint8_t sm[];
    __shared__ ItemCtx X;
    __shared__ float s_invz[kKT];
    __shared__ int abort, next_chunk, s_it;
    if (threadIdx.x == 0) abort = 0;
    hist_init_mbar(sm, tile_rows, hist_warps(MODE));
    uint32_t wseq = 0;
    // this stream's items are handed out one at a time in their (longest
    // first) order
    const int n_items = *count;
    for (;;) {
        __syncthreads();  // every thread has read the previous s_it
        if (threadIdx.x == 0) s_it = atomicAdd(next_item, 1);
        __syncthreads();
        const int it = s_it;
        if (it >= n_items) break;
        const HistItem w = items[list[it]];
        hist_item<NF, MODE>(insts + w.inst, w.p, w.cg, (int64_t)w.kt * kKT, sm, tile_rows, wseq, &abort, X, s_invz,
                            &next_chunk);
    }
}

// Fallback when a part's tile does not fit shared memory (or 3-D rest indices
// exceed the run-end encoding): factors are gathered from global memory
// (L1-cached), rest-axis factors prefetched in register blocks.
__global__ void __launch_bounds__(kHistWarps * 32, 1) k_hist_global(HistArgs A, int G) {
    const LayoutArgs H = pick(A);
    const int p = blockIdx.x / G, cg = blockIdx.x - p * G;
    if (p >= H.P) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.y * kKT + 4 * lane;
    // chunks cg * group_chunks + j * kHistWarps + warp
    for (int j = 0; j < A.group_chunks / kHistWarps; ++j) {
        const int c = p * A.C + cg * A.group_chunks + j * kHistWarps + warp;
        const int32_t p0 = H.chunk_pt[c], p1 = H.chunk_pt[c + 1];
        if (p0 >= p1) continue;
        const int32_t r0 = H.chunk_run[c], r1 = H.chunk_run[c + 1];
        const Flusher flush{A, H, c, p, p0, p1, H.chunk_bin[2 * c], k, load_inv_z(A, k)};
        // the gathered-axis index comes from the sorted order itself (the point
        // words' row field only covers shared-memory tiles)
        const float *wl = H.g_last + k;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        auto wrest = [&](int32_t r) -> float4 {
            if (r >= r1) return zero4;
            const int32_t rest = H.run_rest[r];
            if (A.ndim == 3) {
                const int64_t a0 = rest / H.n1, a1 = rest - a0 * H.n1;
                return mul4(ld4(H.g0 + a0 * A.K_pad + k), ld4(H.g1 + a1 * A.K_pad + k));
            }
            return ld4(H.g0 + (int64_t)rest * A.K_pad + k);
        };
        int32_t cur_key = H.run_bin[r0];
        float4 bacc = zero4;
        for (int32_t rb = r0; rb < r1; rb += kPF) {
            float4 w[kPF];
    #pragma unroll
            for (int u = 0; u < kPF; ++u) w[u] = wrest(rb + u);
            for (int u = 0; u < kPF; ++u) {
                const int32_t r = rb + u;
                if (r >= r1) break;
                float4 acc = zero4;
                for (int32_t q = H.run_start[r]; q < H.run_start[r + 1]; ++q)
                    add4(acc, ld4(wl + (int64_t)(H.perm[q] % H.n_last) * A.K_pad));
                fma4(bacc, w[u], acc);
                const int32_t nk = r + 1 < r1 ? H.run_bin[r + 1] : -1;
                if (nk != cur_key) {
                    flush(cur_key, bacc);
                    bacc = zero4;
                    cur_key = nk;
                }
            }
        }
    }
}

// Prefix-sum tiles of the interval and record streams, once per (part,
// density): thread (p, k) walks the part's rows of the gathered-axis factor
// table, each factor scaled by the density's normaliser 1 / prod_d Z_d, and
// writes the exclusive prefix sums P[0..nrows] (compensated, each P rounded
// once to FP32) so that rows a .. b - 1 sum to P[b] - P[a].  Tile (p, k-tile)
// is one contiguous block of pre_rows x 128 floats, copied as is into the
// histogram kernel's shared memory.  Returns at once when the device chose
// the point stream, whose tile holds the scaled factors themselves.  Loads
// and stores are marked evict-first: the kernel runs beside the contraction,
// whose operands should keep L2.
__device__ __forceinline__ void prefix_tile(const HistArgs &A, const LayoutArgs &H, float *__restrict__ out, int p,
                                            int64_t k) {
    const int64_t row0 = (int64_t)p * H.part_rows;
    const int64_t nrows = min(H.part_rows, H.n_last - row0);
    const float iz = inv_z(A, k);
    const float *src = H.g_last + row0 * A.K_pad + k;
    float *dst = out + ((int64_t)p * (A.K_pad / kKT) + k / kKT) * A.pre_rows * kKT + (k % kKT);
    float sh = 0.f, sl = 0.f;
    constexpr int kAhead = 32;  // rows loaded ahead (the walk is bound by loads in flight)
    for (int64_t a = 0; a < nrows; a += kAhead) {
        float v[kAhead];
#pragma unroll
        for (int u = 0; u < kAhead; ++u) v[u] = a + u < nrows ? __ldcs(src + (a + u) * A.K_pad) : 0.f;
#pragma unroll
        for (int u = 0; u < kAhead; ++u) {
            if (a + u >= nrows) break;
            __stcs(dst + (a + u) * kKT, sh + sl);
            const float x = v[u] * iz;
            const float t = sh + x, bb = t - sh;
            sl += (sh - (t - bb)) + (x - bb);
            sh = t;
        }
    }
    __stcs(dst + nrows * kKT, sh + sl);
}

__global__ void __launch_bounds__(128) k_prefix_tiles(const __grid_constant__ HistArgs A, float *__restrict__ out,
                                                      int gate_stream) {
    if (A.points_only || (gate_stream && A.sel[1] == 0)) return;
    const LayoutArgs &H = A.sel[0] ? A.L1 : A.L0;
    // tiles (p, k-tile) strided over the grid
    const int64_t nkt = A.K_pad / kKT;
    for (int64_t u = blockIdx.x; u < (int64_t)H.P * nkt; u += gridDim.x)
        prefix_tile(A, H, out, (int)(u / nkt), (u % nkt) * kKT + threadIdx.x);
}

// Finish H[k, b]: for every part, the key (part, b) is either empty, summed
// whole by the single chunk that holds it (direct row), or cut by chunk
// boundaries and summed from the partials of the chunks overlapping it (in
// chunk order); parts are added in order.  Two tiles of 128 densities x 8
// bins per 256 threads: warp w takes bin w, each lane four consecutive
// densities of each tile (the two tiles' loads in flight together), so the
// direct rows and partials are read as coalesced 512-byte rows; the tiles go
// to the [K][B] output through shared memory (8 consecutive bins, one
// 32-byte sector, per row).
constexpr int kFinK = 128, kFinB = 8;
constexpr int kFinNK = 2;     // density tiles per CTA: their loads are in flight together
constexpr int kFinMaxP = 96;  // >= parts of any axis: ceil(32767 / kMaxPartRows) = 84
__device__ __forceinline__ void hist_finish_tiles(const HistArgs &A, int64_t kt0, int bt) {
    __shared__ float tile[kFinNK][kFinB][kFinK + 1];
    __shared__ int2 s_cc[kFinMaxP][kFinB];
    const LayoutArgs &H = A.sel[0] ? A.L1 : A.L0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int P = H.P;
    const bool recs = !A.points_only && A.sel[1] == 2;  // record stream: every non-empty group wrote its rows
    // the chunk range of every (part, bin) key of the bin tile; on the record
    // stream that of the part's group of the bin
    for (int e = threadIdx.x; e < P * kFinB; e += blockDim.x) {
        const int p = e / kFinB, bb = e - p * kFinB, b = bt * kFinB + bb;
        s_cc[p][bb] = b >= A.B ? make_int2(-1, -1)
                      : recs   ? H.rec_gch[p * A.GB + b / kRecBinsH]
                               : H.key_chunks[p * A.B + b];
    }
    __syncthreads();
    const int b = bt * kFinB + warp;
    int64_t kq[kFinNK];  // this lane's first density in each tile
    bool live[kFinNK];   // the tile holds densities
#pragma unroll
    for (int t = 0; t < kFinNK; ++t) {
        live[t] = (kt0 + t) * kFinK < A.K;
        kq[t] = (kt0 + t) * kFinK + 4 * lane;
    }
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 total[kFinNK];
#pragma unroll
    for (int t = 0; t < kFinNK; ++t) total[t] = zero;
    if (b < A.B) {
        // four parts at a time: their direct rows (of every tile) in flight
        // together, then added in part order (cut keys from their chunks'
        // partials)
        for (int p0 = 0; p0 < P; p0 += 4) {
            float4 v[4][kFinNK];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int p = p0 + q;
                const int2 cc = p < P ? s_cc[p][warp] : make_int2(-1, -1);
                const float *row = A.direct + ((int64_t)p * A.B + b) * A.K_pad;
#pragma unroll
                for (int t = 0; t < kFinNK; ++t)
                    v[q][t] = (cc.x >= 0 && cc.x == cc.y && live[t]) ? *reinterpret_cast<const float4 *>(row + kq[t])
                                                                     : zero;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int p = p0 + q;
                if (p >= P) break;
                const int2 cc = s_cc[p][warp];
                if (cc.x < 0) continue;
                if (cc.x == cc.y) {
#pragma unroll
                    for (int t = 0; t < kFinNK; ++t) add4(total[t], v[q][t]);
                    continue;
                }
                // the partials of the chunks holding the key, two chunks'
                // loads (of every tile) in flight together, added in chunk order
                float4 sum[kFinNK];
#pragma unroll
                for (int t = 0; t < kFinNK; ++t) sum[t] = zero;
                const int32_t gr = p * A.GB + b / kRecBinsH, key = p * A.B + b;
                for (int c0 = cc.x; c0 <= cc.y; c0 += 2) {
                    float4 pv[2][kFinNK];
                    bool use[2];
#pragma unroll
                    for (int q2 = 0; q2 < 2; ++q2) {
                        const int c = c0 + q2;
                        use[q2] = false;
#pragma unroll
                        for (int t = 0; t < kFinNK; ++t) pv[q2][t] = zero;
                        if (c > cc.y) continue;
                        const float *row;
                        if (recs) {
                            if (H.rec_chunk[c] >= H.rec_chunk[c + 1]) continue;
                            const int side = H.rec_chunk_grp[2 * c] == gr ? 0 : 1;
                            row = A.part + (((int64_t)c * 2 + side) * kRecBinsH + b % kRecBinsH) * A.K_pad;
                        } else {
                            if (H.chunk_pt[c] >= H.chunk_pt[c + 1]) continue;
                            const int side = H.chunk_bin[2 * c] == key ? 0 : 1;
                            row = A.part + ((int64_t)c * 2 + side) * A.K_pad;
                        }
#pragma unroll
                        for (int t = 0; t < kFinNK; ++t)
                            if (live[t]) pv[q2][t] = *reinterpret_cast<const float4 *>(row + kq[t]);
                        use[q2] = true;
                    }
#pragma unroll
                    for (int q2 = 0; q2 < 2; ++q2)
                        if (use[q2])
#pragma unroll
                            for (int t = 0; t < kFinNK; ++t) add4(sum[t], pv[q2][t]);
                }
#pragma unroll
                for (int t = 0; t < kFinNK; ++t) add4(total[t], sum[t]);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < kFinNK; ++t) {
        float *row = tile[t][warp] + 4 * lane;
        row[0] = total[t].x;
        row[1] = total[t].y;
        row[2] = total[t].z;
        row[3] = total[t].w;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kFinNK * kFinK * kFinB; e += blockDim.x) {
        const int t = e / (kFinK * kFinB), r = e - t * (kFinK * kFinB);
        const int kk = r / kFinB, bb = r - kk * kFinB;
        const int64_t kr = (kt0 + t) * kFinK + kk;
        const int bo = bt * kFinB + bb;
        if (kr < A.K && bo < A.B) A.hist[kr * A.B + bo] = tile[t][bb][kk];
    }
}

__global__ void __launch_bounds__(256, 3) k_hist_finish(const __grid_constant__ HistArgs A) {
    pdl_trigger();
    pdl_wait();
    hist_finish_tiles(A, (int64_t)blockIdx.x * kFinNK, blockIdx.y);
}

// Batched finish: items[i] = (instance, density tile, bin tile).
__global__ void __launch_bounds__(256, 3) k_hist_finish_batched(const HistArgs *__restrict__ insts, const int4 *__restrict__ items) {
    const int4 it = items[blockIdx.x];
    hist_finish_tiles(insts[it.x], (int64_t)it.y * kFinNK, it.z);
}

}  // namespace

// Chunks per part: groups of kGroupChunks chunks, as many groups (1..16) as
// give chunks of about 1536 points when the gathered axis is cut into P
// parts.  A launch then picks how many groups one CTA serves.
int vup_hist_chunks_for(int64_t N, int P) {
    const double per_group = (double)kGroupChunks * 1536.0;
    int64_t S = (int64_t)llround((double)N / ((double)std::max(P, 1) * per_group));
    S = std::max<int64_t>(1, std::min<int64_t>(16, S));
    return (int)(S * kGroupChunks);
}

// Record chunks per part: a quarter of the point chunks (records are several
// times fewer than intervals), in whole groups of kGroupChunks.
int vup_hist_rec_chunks_for(int n_chunks) {
    return kGroupChunks * std::max(1, n_chunks / kGroupChunks / 4);
}

// Parts of a gathered axis of n_last rows (one 64-density tile each) for a
// bin count; one part when the (part, bin) key space would exceed the sort.
int vup_hist_parts_for(int64_t n_last, int n_bins) {
    int P = (int)ceil_div64(n_last, kMaxPartRows);
    if ((int64_t)P * n_bins > 32768) P = 1;
    return P;
}

// Arguments of the histogram kernels for one grid; `rows` receives the
// largest shared-memory tile (rows of one part of a gathered axis).
static HistArgs hist_args_for(vup_grid g, int64_t K, float *hist, int64_t &rows, int &P_max,
                              const float *ftab = nullptr) {
    const int64_t K_pad = ceil_div64(K, 128) * 128;
    const int nd = g->ndim;
    const float *ft = ftab ? ftab : (const float *)g->ftab.p;
    auto tab = [&](int axis) {
        int64_t off = 0;
        for (int q = 0; q < axis; ++q) off += g->n[q] * K_pad;
        return ft + off;
    };
    HistArgs A{};
    A.group_chunks = kGroupChunks;
    rows = 0;
    P_max = 1;
    for (int l = 0; l < 2; ++l) {
        const auto &HL = g->hl[l < g->n_layouts ? l : 0];
        LayoutArgs &La = l == 0 ? A.L0 : A.L1;
        La.hpt = HL.hpt;
        La.perm = HL.perm;
        La.run_start = HL.run_start;
        La.run_rest = HL.run_rest;
        La.run_bin = HL.run_bin;
        La.chunk_pt = HL.chunk_pt;
        La.chunk_run = HL.chunk_run;
        La.chunk_bin = HL.chunk_bin;
        La.koff = HL.koff;
        La.key_chunks = HL.key_chunks;
        La.ipt = HL.ipt;
        La.iv_rest = HL.iv_rest;
        La.chunk_iv = HL.chunk_iv;
        La.rec = (const uint4 *)g->hl[0].rec.p;  // the built layout's arrays
        La.rec_rest = (const int32_t *)g->hl[0].rec_rest.p;
        La.rec_goff = (const int32_t *)g->hl[0].rec_goff.p;
        La.rec_gch = (const int2 *)g->hl[0].rec_gch.p;
        La.rec_chunk = g->hl[0].rec_chunk;
        La.rec_chunk_grp = g->hl[0].rec_chunk_grp;
        La.g_last = tab(HL.last_axis);
        if (nd == 3) {
            La.g0 = tab(0);
            La.g1 = tab(1);
            La.n1 = g->n[1];
            La.n0 = g->n[0];
        } else {
            La.g0 = tab(HL.last_axis == 1 ? 0 : 1);
            La.g1 = nullptr;
            La.n1 = 1;
            La.n0 = g->n[HL.last_axis == 1 ? 0 : 1];
        }
        La.n_last = HL.n_last;
        La.part_rows = HL.part_rows;
        La.P = HL.P;
        rows = std::max(rows, HL.part_rows);
        P_max = std::max(P_max, HL.P);
    }
    A.sel = g->hist_sel;
    A.GB = (int)ceil_div64(g->B, kRecBinsH);
    A.rec_sets = 1;
    A.C_rec = g->n_chunks_rec;
    A.ds = (const DensStats *)g->dstats.p;
    A.ndim = nd;
    A.K = K;
    A.K_pad = K_pad;
    A.B = g->B;
    A.C = g->n_chunks;
    A.hist = hist;
    A.part = (float *)g->hist_part.p;
    A.direct = (float *)g->hist_direct.p;
    A.dstatus = g->dstatus;
    return A;
}

bool vup_hist_prefix(vup_grid g, int64_t K, cudaStream_t s) {
    if (!vup_hist_tile_fits(g)) return false;
    int64_t rows;
    int P_max;
    HistArgs A = hist_args_for(g, K, nullptr, rows, P_max);
    A.pre_rows = rows + 1;
    VUP_PROF("hist_prefix", s, 1);
    k_prefix_tiles<<<(unsigned)(P_max * (A.K_pad / 128)), 128, 0, s>>>(A, (float *)g->hist_prefix.p, 0);
    return cudaGetLastError() == cudaSuccess;
}

bool vup_hist_rest_staged(const vup_grid_s *g) {
    if (g->ndim != 3 || g->hl[0].last_axis != 2 || g->n[0] > 512 || g->n[1] > 4096) return false;
    const size_t rest_bytes = (size_t)(g->n[0] + g->n[1]) * kKT * sizeof(float);
    return hist_smem_bytes(g->hl[0].part_rows, hist_warps(4)) + rest_bytes <= 220 * 1024;
}

vup_status vup_hist_fused(vup_grid g, int64_t K, float *hist, cudaStream_t s, const float *ftab,
                          bool points_only, cudaEvent_t keys_ready, bool prefix_ready) {
    const int nd = g->ndim;
    int64_t rows;
    int P_max;
    HistArgs A = hist_args_for(g, K, hist, rows, P_max, ftab);
    const size_t smem = hist_smem_bytes(rows);
    // run-end words encode the rest index in 21 bits (3-D: a0 < 512, a1 < 4096)
    const bool coded = nd == 2 || (g->n[0] <= 512 && g->n[1] <= 4096);
    const bool in_smem = smem <= 220 * 1024 && coded;
    // 3-D point stream: both rest-axis factor tiles in shared memory when they fit beside the tile
    const size_t rest_bytes = nd == 3 ? (size_t)(g->n[0] + g->n[1]) * kKT * sizeof(float) : 0;
    A.rest_n0 = nd == 3 ? g->n[0] : 0;
    A.rest_smem = in_smem && vup_hist_rest_staged(g);
    // the global-memory fallback walks points whatever the device chose
    points_only = points_only || !in_smem;
    A.points_only = points_only ? 1 : 0;
    // items: G groups of C / G chunks per part, G dividing C / kGroupChunks,
    // chosen for the fewest idle SM slots in the last wave (one CTA per SM)
    const int S = A.C / kGroupChunks, nkt = (int)ceil_div64(K, kKT), sms = vup_num_sms();
    int G = S;
    double best = -1.0;
    for (int gg = S; gg >= 1; --gg) {
        if (S % gg) continue;
        const int64_t items = (int64_t)P_max * gg * nkt;
        const double eff = (double)items / (double)(ceil_div64(items, sms) * sms);
        if (eff > best + 0.02) {
            best = eff;
            G = gg;
        }
    }
    A.group_chunks = A.C / G;
    const int n_items = P_max * G * nkt;
    // record stream: S items per part, each a range of its record chunks, S for
    // the fullest last wave
    int Sr = 1;
    {
        double best_r = -1.0;
        for (int ss = 1; ss <= std::max(1, A.C_rec / hist_warps(3)); ++ss) {  // at least a chunk per warp
            const int64_t items = (int64_t)P_max * ss * nkt;
            const double eff = (double)items / (double)(ceil_div64(items, sms) * sms);
            if (eff > best_r + 0.02) {
                best_r = eff;
                Sr = ss;
            }
        }
    }
    A.rec_sets = Sr;
    const int n_items_rec = P_max * Sr * nkt;
    if (in_smem && !points_only && !ftab) {
        // prefix-sum tiles for the interval and record streams (the kernel
        // returns at once when the device chose the point stream)
        A.prefix = (const float *)g->hist_prefix.p;
        A.pre_rows = rows + 1;
        if (!prefix_ready) {
            VUP_PROF("hist_prefix", s, 1);
            k_prefix_tiles<<<(unsigned)(P_max * (A.K_pad / 128)), 128, 0, s>>>(A, (float *)g->hist_prefix.p, 1);
            VUP_CHECK_LAUNCH();
        }
    }
    {
        VUP_PROF("hist_segmented", s, in_smem && !points_only ? 3 : 1);
        if (in_smem) {
            auto launch = [&](auto kern, int gg, int items, int mode) -> vup_status {
                const size_t sm_bytes = hist_smem_bytes(rows, hist_warps(mode)) + (mode == 4 ? rest_bytes : 0);
                VUP_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_bytes));
                VUP_CHECK_CUDA(launch_pdl(kern, dim3(items), dim3(hist_warps(mode) * 32), sm_bytes, s, A, rows,
                                          P_max, gg, items));
                return VUP_OK;
            };
            vup_status st;
            if (!points_only) {  // the record stream first: it needs no key sort
                // 16 warps when the rest-factor rows (of either layout) fit well in L2
                int64_t rest_rows = 0;
                for (int l = 0; l < g->n_layouts; ++l) rest_rows = std::max(rest_rows, g->N / g->hl[l].n_last);
                if (nd == 3) rest_rows = g->n[0] + g->n[1];
                const bool l2_rest = (double)rest_rows * A.K_pad * 4.0 <= 96.0 * 1024 * 1024;
                if (l2_rest)
                    st = nd == 3 ? launch(k_hist_smem<2, 3>, Sr, n_items_rec, 3)
                                 : launch(k_hist_smem<1, 3>, Sr, n_items_rec, 3);
                else
                    st = nd == 3 ? launch(k_hist_smem<2, 2>, Sr, n_items_rec, 2)
                                 : launch(k_hist_smem<1, 2>, Sr, n_items_rec, 2);
                if (st != VUP_OK) return st;
            }
            if (keys_ready) VUP_CHECK_CUDA(cudaStreamWaitEvent(s, keys_ready, 0));
            st = nd == 3 ? (A.rest_smem ? launch(k_hist_smem<2, 4>, G, n_items, 4)
                                        : launch(k_hist_smem<2, 0>, G, n_items, 0))
                         : launch(k_hist_smem<1, 0>, G, n_items, 0);
            if (st != VUP_OK) return st;
            if (!points_only) {
                st = nd == 3 ? launch(k_hist_smem<2, 1>, G, n_items, 1) : launch(k_hist_smem<1, 1>, G, n_items, 1);
                if (st != VUP_OK) return st;
            }
        } else {
            if (keys_ready) VUP_CHECK_CUDA(cudaStreamWaitEvent(s, keys_ready, 0));
            dim3 grd((unsigned)(P_max * G), (unsigned)nkt);
            k_hist_global<<<grd, kHistWarps * 32, 0, s>>>(A, G);
            VUP_CHECK_LAUNCH();
        }
    }
    VUP_PROF("hist_fixup", s, 1);
    dim3 fg((unsigned)ceil_div64(K, kFinK * kFinNK), (unsigned)ceil_div64(g->B, kFinB));
    VUP_CHECK_CUDA(launch_pdl(k_hist_finish, fg, dim3(32 * kFinB), 0, s, A));
    return VUP_OK;
}

bool vup_hist_tile_fits(vup_grid g) {
    const bool coded = g->ndim == 2 || (g->n[0] <= 512 && g->n[1] <= 4096);
    for (int l = 0; l < g->n_layouts; ++l)
        if (hist_smem_bytes(g->hl[l].part_rows) > 220 * 1024) return false;
    return coded;
}

// A 2-D grid whose every part fits the shared-memory tile.
bool vup_hist_batchable(vup_grid g) {
    if (g->ndim != 2) return false;
    for (int l = 0; l < g->n_layouts; ++l)
        if (hist_smem_bytes(g->hl[l].part_rows) > 220 * 1024) return false;
    return true;
}

// Batched histograms of n 2-D instances: one persistent launch over every
// instance's (part, chunk group, density tile) items, longest first, and one
// finishing launch.
struct HistPlan {
    DevBuf args, items, fitems, ctr;  // ctr: next item of each stream's launch, then each stream's item count
    DevBuf lists;                     // [3][n_items] each stream's items (k_hist_split_items)
    int n_inst = 0, n_items = 0, n_fitems = 0;
    int64_t rows = 0;
};

vup_status vup_hist_plan(int n, const vup_grid *gs, const int64_t *Ks, float *const *hists, void **out) {
    std::vector<HistArgs> args(n);
    std::vector<std::pair<int64_t, HistItem>> work;
    std::vector<int4> fin;
    int64_t rows_max = 0;
    for (int i = 0; i < n; ++i) {
        int64_t rows;
        int P_max;
        args[i] = hist_args_for(gs[i], Ks[i], hists[i], rows, P_max);
        if (!hists[i]) continue;
        rows_max = std::max(rows_max, rows);
        args[i].group_chunks = kGroupChunks;
        const int G = args[i].C / kGroupChunks;
        args[i].rec_sets = G;  // record stream: item cg takes the cg-th of G ranges of the part's record chunks
        const int64_t nkt = ceil_div64(Ks[i], kKT);
        // cost of one item: points per chunk x densities per tile
        const int64_t cost = gs[i]->N / std::max<int64_t>(1, (int64_t)P_max * args[i].C);
        for (int p = 0; p < P_max; ++p)
            for (int cg = 0; cg < G; ++cg)
                for (int64_t kt = 0; kt < nkt; ++kt) work.push_back({cost, HistItem{i, p, cg, (int32_t)kt}});
        for (int64_t kb = 0; kb < ceil_div64(Ks[i], kFinK * kFinNK); ++kb)
            for (int bt = 0; bt < (int)ceil_div64(gs[i]->B, kFinB); ++bt) fin.push_back(make_int4(i, (int)kb, bt, 0));
    }
    std::stable_sort(work.begin(), work.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::vector<HistItem> items(work.size());
    for (size_t q = 0; q < work.size(); ++q) items[q] = work[q].second;
    HistPlan *P = new HistPlan();
    P->n_inst = n;
    P->n_items = (int)items.size();
    P->n_fitems = (int)fin.size();
    P->rows = rows_max;
    vup_status st;
    if ((st = devbuf_reserve(P->args, sizeof(HistArgs) * n)) != VUP_OK ||
        (st = devbuf_reserve(P->items, sizeof(HistItem) * std::max<size_t>(1, items.size()))) != VUP_OK ||
        (st = devbuf_reserve(P->fitems, sizeof(int4) * std::max<size_t>(1, fin.size()))) != VUP_OK ||
        (st = devbuf_reserve(P->ctr, sizeof(int) * 6)) != VUP_OK ||
        (st = devbuf_reserve(P->lists, sizeof(int32_t) * 3 * std::max<size_t>(1, items.size()))) != VUP_OK) {
        devbuf_free(P->args);
        devbuf_free(P->items);
        devbuf_free(P->fitems);
        devbuf_free(P->ctr);
        devbuf_free(P->lists);
        delete P;
        return st;
    }
    VUP_CHECK_CUDA(cudaMemcpy(P->args.p, args.data(), sizeof(HistArgs) * n, cudaMemcpyHostToDevice));
    VUP_CHECK_CUDA(cudaMemcpy(P->items.p, items.data(), sizeof(HistItem) * items.size(), cudaMemcpyHostToDevice));
    VUP_CHECK_CUDA(cudaMemcpy(P->fitems.p, fin.data(), sizeof(int4) * fin.size(), cudaMemcpyHostToDevice));
    // the largest tile any plan may use, so that graphs of earlier plans stay launchable
    VUP_CHECK_CUDA(
        cudaFuncSetAttribute(k_hist_batched<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    VUP_CHECK_CUDA(
        cudaFuncSetAttribute(k_hist_batched<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    VUP_CHECK_CUDA(
        cudaFuncSetAttribute(k_hist_batched<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    *out = P;
    return VUP_OK;
}

void vup_hist_plan_free(void *plan) {
    HistPlan *P = (HistPlan *)plan;
    if (!P) return;
    devbuf_free(P->args);
    devbuf_free(P->items);
    devbuf_free(P->fitems);
    devbuf_free(P->ctr);
    devbuf_free(P->lists);
    delete P;
}

vup_status vup_hist_batched(void *plan, cudaStream_t s) {
    const HistPlan *P = (const HistPlan *)plan;
    if (P->n_items == 0) return VUP_OK;
    const size_t smem = hist_smem_bytes(P->rows);
    if (smem > 220 * 1024) return VUP_ERR_UNSUPPORTED;
    {
        VUP_PROF("hist_segmented_batched", s, 4);
        const int grid = std::max(1, std::min(P->n_items, vup_num_sms()));
        int *ctr = (int *)P->ctr.p, *counts = ctr + 3;
        const int32_t *lists = (const int32_t *)P->lists.p;
        const HistArgs *args = (const HistArgs *)P->args.p;
        const HistItem *items = (const HistItem *)P->items.p;
        VUP_CHECK_CUDA(cudaMemsetAsync(ctr, 0, 3 * sizeof(int), s));
        const size_t split_smem = P->n_inst <= kSplitStaged ? (size_t)P->n_inst : 0;
        k_hist_split_items<<<1, kSplitThreads, split_smem, s>>>(args, P->n_inst, items, P->n_items,
                                                                (int32_t *)P->lists.p, counts);
        VUP_CHECK_LAUNCH();
        k_hist_batched<1, 0><<<grid, kHistWarps * 32, smem, s>>>(args, items, lists, counts, P->rows, ctr);
        VUP_CHECK_LAUNCH();
        k_hist_batched<1, 1><<<grid, kHistWarps * 32, smem, s>>>(args, items, lists + P->n_items, counts + 1,
                                                                 P->rows, ctr + 1);
        VUP_CHECK_LAUNCH();
        k_hist_batched<1, 2><<<grid, hist_warps(2) * 32, hist_smem_bytes(P->rows, hist_warps(2)), s>>>(
            args, items, lists + 2 * (size_t)P->n_items, counts + 2, P->rows, ctr + 2);
        VUP_CHECK_LAUNCH();
    }
    VUP_PROF("hist_fixup_batched", s, 1);
    k_hist_finish_batched<<<P->n_fitems, 32 * kFinB, 0, s>>>((const HistArgs *)P->args.p,
                                                             (const int4 *)P->fitems.p);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}
