// Supplied-weights VUP: the input probability matrix is given explicitly
// (N x K in the paper's Eq. VUP, stored here row-major as W[K][N]) and is
// streamed once from HBM.  Every grid point's weight is multiplied into the
// moment sums and added into its output bin (the one-hot model matrix of
// Eq. MUP applied to each column).  The roofline is the W read: 4 bytes per
// distribution-point.  Forms: the bin-sorted block walk k_weights_sorted
// (B <= 1024, rows of W 16-byte aligned; the blocks sorted once per model by
// k_wsort_blocks), else k_weights_t (a row per lane, shared-memory atomics;
// B <= 1024) or k_weights<RB> (larger B), each finished by
// k_weights_finish.
#include "vup_internal.cuh"
#include "vup_async.cuh"

#include <algorithm>

namespace {

constexpr int kThreads = 256;

// Every form below sums each thread's moment terms in short FP32 runs folded
// into TwoSum pairs (two_sum_acc), so that a long point range keeps about
// FP32-squared accuracy.

template <int RB>
__global__ void __launch_bounds__(kThreads) k_weights(const float *__restrict__ W, int64_t K, int64_t N,
                                                      const float *__restrict__ z32,
                                                      const int32_t *__restrict__ bins, int B, int64_t n_split,
                                                      double *__restrict__ mpart, float *__restrict__ hpart) {
    extern __shared__ float sh[];  // [RB][B]
    __shared__ double red[RB][4][kThreads / 32];
    const int64_t split = blockIdx.x;
    const int64_t k0 = (int64_t)blockIdx.y * RB;
    for (int e = threadIdx.x; e < RB * B; e += blockDim.x) sh[e] = 0.f;
    __syncthreads();
    // rows past K re-read row K-1 and are never stored, so that every row's
    // load is unconditional and all RB loads of a column are in flight at once
    const float *wrow[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) wrow[r] = W + min(k0 + r, K - 1) * N;
    // column range of this split, in float4 units (rows of W are 16-byte
    // aligned only when N is a multiple of 4; otherwise every column goes
    // through the scalar loop below)
    const int64_t n4 = (N % 4 == 0 && (reinterpret_cast<uintptr_t>(W) & 15) == 0) ? N / 4 : 0;
    const int64_t per = (n4 + n_split - 1) / n_split;
    const int64_t c0 = split * per, c1 = min(n4, c0 + per);
    float m[RB][4], ml[RB][4];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int j = 0; j < 4; ++j) m[r][j] = ml[r][j] = 0.f;
#pragma unroll 2
    for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        float4 w[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) w[r] = __ldcs(reinterpret_cast<const float4 *>(wrow[r]) + c);
        const float4 z = *reinterpret_cast<const float4 *>(z32 + c * 4);
        const int4 b = *reinterpret_cast<const int4 *>(bins + c * 4);
        const float zz[4] = {z.x, z.y, z.z, z.w};
        const int bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const float ww[4] = {w[r].x, w[r].y, w[r].z, w[r].w};
            float s4[4] = {0.f, 0.f, 0.f, 0.f};  // the column's four points, then folded
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float p = zz[q];
                float t = ww[q] * p;
                s4[0] += t;
                t *= p; s4[1] += t;
                t *= p; s4[2] += t;
                t *= p; s4[3] += t;
                atomicAdd(&sh[r * B + bb[q]], ww[q]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) two_sum_acc(m[r][j], ml[r][j], s4[j]);
        }
    }
    // columns not covered by the float4 loop, split evenly
    {
        const int64_t rem = N - n4 * 4;
        const int64_t per1 = (rem + n_split - 1) / n_split;
        const int64_t i0 = n4 * 4 + split * per1, i1 = min(N, i0 + per1);
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const float p = z32[i];
            const int bq = bins[i];
            for (int r = 0; r < RB; ++r) {
                const float w = wrow[r][i];
                float t = w * p;
                two_sum_acc(m[r][0], ml[r][0], t);
                t *= p; two_sum_acc(m[r][1], ml[r][1], t);
                t *= p; two_sum_acc(m[r][2], ml[r][2], t);
                t *= p; two_sum_acc(m[r][3], ml[r][3], t);
                atomicAdd(&sh[r * B + bq], w);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double v = (double)m[r][j] + (double)ml[r][j];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[r][j][warp] = v;
        }
    __syncthreads();
    if (threadIdx.x < RB * 4) {
        const int r = threadIdx.x >> 2, j = threadIdx.x & 3;
        double v = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) v += red[r][j][w];
        if (k0 + r < K) mpart[(split * K + k0 + r) * 4 + j] = v;
    }
    for (int e = threadIdx.x; e < RB * B; e += blockDim.x) {
        const int r = e / B, b = e - r * B;
        if (k0 + r < K) hpart[(split * K + k0 + r) * B + b] = sh[e];
    }
}

// Row-per-lane form for B <= 1024: lane l of every warp owns row k0 + l, so
// the 32 shared-memory atomics of one instruction go to 32 different rows'
// histograms (row stride B + 1: 32 different banks) and never collide.  Each
// lane streams 64 contiguous bytes of its row per step; the z and bin values
// of a step are the same for every lane (broadcast loads).  Warps split the
// CTA's point range; the CTA's 32 histograms live in shared memory.
constexpr int kRowsT = 32;
constexpr int kPtsT = 16;   // points per lane per step
__global__ void __launch_bounds__(kThreads) k_weights_t(const float *__restrict__ W, int64_t K, int64_t N,
                                                        const float *__restrict__ z32,
                                                        const int32_t *__restrict__ bins, int B, int64_t n_split,
                                                        double *__restrict__ mpart, float *__restrict__ hpart) {
    extern __shared__ float sh[];  // [kRowsT][B + 1]
    __shared__ double red[kThreads / 32][kRowsT][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t split = blockIdx.x;
    const int64_t k0 = (int64_t)blockIdx.y * kRowsT;
    const int ld = B + 1;
    for (int e = threadIdx.x; e < kRowsT * ld; e += blockDim.x) sh[e] = 0.f;
    __syncthreads();
    const float *wrow = W + min(k0 + lane, K - 1) * N;  // rows past K are never stored
    float *hrow = sh + lane * ld;
    // moments: a step's 16 points are summed on their own, then folded into
    // the running TwoSum pairs
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, l0 = 0.f, l1 = 0.f, l2 = 0.f, l3 = 0.f;
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
    auto point = [&](float w, float p, int b) {
        float t = w * p;
        t0 += t;
        t *= p;
        t1 += t;
        t *= p;
        t2 += t;
        t *= p;
        t3 += t;
        atomicAdd(hrow + b, w);
    };
    auto fold = [&]() {
        two_sum_acc(m0, l0, t0);
        two_sum_acc(m1, l1, t1);
        two_sum_acc(m2, l2, t2);
        two_sum_acc(m3, l3, t3);
        t0 = t1 = t2 = t3 = 0.f;
    };
    // vector steps of kPtsT points (rows 16-byte aligned only when N % 4 == 0)
    const bool vec = N % 4 == 0 && (reinterpret_cast<uintptr_t>(W) & 15) == 0;
    const int64_t n_steps = vec ? N / kPtsT : 0;
    const int64_t per = (n_steps + n_split - 1) / n_split;
    const int64_t s0 = split * per, s1 = min(n_steps, s0 + per);
    for (int64_t st = s0 + warp; st < s1; st += kThreads / 32) {
        const int64_t i = st * kPtsT;
        float4 w[4], z[4];
        int4 b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = __ldcs(reinterpret_cast<const float4 *>(wrow + i) + q);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            z[q] = *reinterpret_cast<const float4 *>(z32 + i + 4 * q);
            b[q] = *reinterpret_cast<const int4 *>(bins + i + 4 * q);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            point(w[q].x, z[q].x, b[q].x);
            point(w[q].y, z[q].y, b[q].y);
            point(w[q].z, z[q].z, b[q].z);
            point(w[q].w, z[q].w, b[q].w);
        }
        fold();
    }
    // points not covered by the vector steps, split evenly
    {
        const int64_t rem = N - n_steps * kPtsT;
        const int64_t per1 = (rem + n_split - 1) / n_split;
        const int64_t i0 = n_steps * kPtsT + split * per1, i1 = min(N, i0 + per1);
        int64_t n_pt = 0;
        for (int64_t i = i0 + warp; i < i1; i += kThreads / 32) {
            point(wrow[i], z32[i], bins[i]);
            if (++n_pt == kPtsT) {
                fold();
                n_pt = 0;
            }
        }
        fold();
    }
    red[warp][lane][0] = (double)m0 + (double)l0;
    red[warp][lane][1] = (double)m1 + (double)l1;
    red[warp][lane][2] = (double)m2 + (double)l2;
    red[warp][lane][3] = (double)m3 + (double)l3;
    __syncthreads();
    if (threadIdx.x < kRowsT * 4) {
        const int r = threadIdx.x >> 2, j = threadIdx.x & 3;
        double v = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) v += red[q][r][j];
        if (k0 + r < K) mpart[(split * K + k0 + r) * 4 + j] = v;
    }
    for (int e = threadIdx.x; e < kRowsT * B; e += blockDim.x) {
        const int r = e / B, bb = e - r * B;
        if (k0 + r < K) hpart[(split * K + k0 + r) * B + bb] = sh[r * ld + bb];
    }
}

// Sorted-block walk (B <= 1024, rows of W 16-byte aligned).  The grid's
// points are cut into blocks of kWBlock; within a block they are sorted by
// bin once per model (wsort_*), and warp w walks sorted positions
// [32 w, 32 w + 32) of every block.  A CTA owns 32 rows of W (lane l: row
// k0 + l) and a range of blocks; each block's 32 x 256 tile of W is staged in
// shared memory by bulk copies (cp.async.bulk, one per row, issued by warp 0
// and completing on the stage's mbarrier; two stages) together with the
// block's sorted words and z values.  Rows are padded to 260 floats: a warp
// reading one column of 32 rows touches 8 banks (a 4-way conflict; rows
// copied in 16-byte units cannot spread one column over more than 8).  A
// bin's points (a run) are summed in a register and added once to the lane's
// histogram row in shared memory.  A run inside one slice has one writer and
// is added by a plain read-modify-write; a run that crosses a slice edge is
// summed per slice into the warp's own scratch columns of the row and added
// to its bin with a shared-memory atomic after the walk.  The moments are
// summed per block in FP32 and across blocks as TwoSum pairs.  The histogram
// rows hold at most ~64 blocks' contributions per bin (column splits are
// sized for that), the partial rows are summed as FP32 TwoSum pairs.
constexpr int kWBlock = 256;
constexpr int kWLd = kWBlock + 4;       // padded tile row (floats)
constexpr int kWRows = 32;
constexpr int kWMaxBlocksPerCta = 64;   // bounds each FP32 histogram sum
constexpr int kWWarps = 8;              // warp slices per block
constexpr int kWThreads = kWWarps * 32;
constexpr int kWSlice = kWBlock / kWWarps;
// Histogram row of a lane: bins 0..B-1, then a spare column B (the flush
// before a slice's first run lands there), the warps' head columns B+1+w (a
// run continued from the previous slice) and tail columns B+1+kWWarps+w (a
// run continuing into the next slice); odd row length, so that the 32 rows'
// entries of one column fall in 32 banks.
constexpr int kWExtraCols = 1 + 2 * kWWarps;
__host__ __device__ constexpr int w_hist_ld(int B) { return (B + kWExtraCols) | 1; }
// two words per sorted position: the byte offset of its column in a tile
// row (pt[t]), and the byte offset of its histogram entry plus 1 if it is the
// first position of its run (pt[kWBlock + t]); a run that continues into the
// next slice names the warp's tail column.  Positions past the grid's end:
// the zero column, word 0.  fix[w] / fix[kWWarps + w]: the bin of slice w's
// head / tail run with bit 15 set when that run crosses the slice's start /
// end.
constexpr uint32_t kWFillerCol = (uint32_t)kWBlock * 4u;
constexpr int kWFix = 2 * kWWarps;
constexpr uint16_t kWCross = 0x8000u;
struct WStage {
    float tile[kWRows][kWLd];  // column kWBlock is zero (the fillers' column)
    uint32_t pt[2 * kWBlock];
    float z[kWBlock];  // z = y / s_abs; the walk forms z^2..z^4 (as the sort kernel would)
    uint16_t fix[kWFix];
};

using namespace vup_async;


template <int STAGES, int MINB>
__global__ void __launch_bounds__(kWThreads, MINB)
k_weights_sorted(const float *__restrict__ W, int64_t K, int64_t N, const uint32_t *__restrict__ wpt,
                 const float *__restrict__ wz, const uint16_t *__restrict__ wfix, int B, int64_t n_split,
                 double *__restrict__ mpart, float *__restrict__ hpart, int *dstatus) {
    extern __shared__ __align__(16) uint8_t wsm[];
    __shared__ uint64_t full[STAGES];
    __shared__ int abort_flag;
    WStage *st = reinterpret_cast<WStage *>(wsm);
    float *H = reinterpret_cast<float *>(wsm + sizeof(WStage) * STAGES);  // [kWRows][ld]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ld = w_hist_ld(B);
    const int64_t k0 = (int64_t)blockIdx.y * kWRows;
    const int64_t n_blk = (N + kWBlock - 1) / kWBlock;
    const int64_t split = blockIdx.x;
    const int64_t c_lo = split * n_blk / n_split, c_hi = (split + 1) * n_blk / n_split;
    for (int e = threadIdx.x; e < kWRows * ld; e += blockDim.x) H[e] = 0.f;
    for (int e = threadIdx.x; e < STAGES * kWRows; e += blockDim.x) st[e / kWRows].tile[e % kWRows][kWBlock] = 0.f;
    if (threadIdx.x == 0) {
        for (int q = 0; q < STAGES; ++q) mbar_init(&full[q], kWWarps);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // stage block c into buffer b (every warp: lanes 0-3 of warp w copy rows
    // 4 w .. 4 w + 3 of W, rows past K re-reading row K - 1, never stored;
    // warp 0 also the block's sorted words, z values and crossing runs); each
    // warp adds its bytes to full[b] and arrives once
    auto stage = [&](int64_t c, int b) {
        WStage &S = st[b];
        const int64_t col0 = c * kWBlock;
        const uint32_t row_bytes = (uint32_t)min((int64_t)kWBlock, N - col0) * 4u;
        constexpr uint32_t meta = (uint32_t)(sizeof(WStage::pt) + sizeof(WStage::z) + sizeof(WStage::fix));
        constexpr int rows_per_warp = kWRows / kWWarps;
        if (lane == 0) mbar_expect_tx(&full[b], rows_per_warp * row_bytes + (warp == 0 ? meta : 0u));
        __syncwarp();
        if (lane < rows_per_warp) {
            const int r = warp * rows_per_warp + lane;
            bulk_g2s(&S.tile[r][0], W + min(k0 + r, K - 1) * N + col0, row_bytes, &full[b]);
        }
        if (warp == 0 && lane == 0) {
            bulk_g2s(S.pt, wpt + c * 2 * kWBlock, (uint32_t)sizeof(S.pt), &full[b]);
            bulk_g2s(S.z, wz + c * kWBlock, (uint32_t)sizeof(S.z), &full[b]);
            bulk_g2s(S.fix, wfix + c * kWFix, (uint32_t)sizeof(S.fix), &full[b]);
        }
    };
    int64_t issued = 0;  // blocks staged so far
    bool stop = false;   // a wait expired (the same value in every thread)
    for (int q = 0; q < STAGES - 1 && c_lo + q < c_hi; ++q, ++issued) stage(c_lo + q, q);
    // per-row moment sums across blocks: FP32 pairs (sum, compensation)
    // updated by TwoSum (Knuth), exact to about FP32 squared; one FP64
    // conversion per CTA at the end
    float mhi[4] = {0.f, 0.f, 0.f, 0.f}, mlo[4] = {0.f, 0.f, 0.f, 0.f};
    const float *hrow = H + lane * ld;
    const uint32_t hbase = (uint32_t)__cvta_generic_to_shared(hrow), hbase_m1 = hbase - 1u;
    for (int64_t c = c_lo; c < c_hi; ++c) {
        const int b = (int)((c - c_lo) % STAGES);
        // keep STAGES - 1 blocks in flight: issue block c + STAGES - 1 (its
        // buffer was last read in iteration c - 1, before that iteration's
        // closing barrier), then wait for block c.  After an expired wait
        // nothing more is issued or walked; every thread still meets the
        // closing barriers, and the copies in flight are drained below.
        if (!stop && c + STAGES - 1 < c_hi) {
            stage(c + STAGES - 1, (int)((c + STAGES - 1 - c_lo) % STAGES));
            ++issued;
        }
        const bool ready = mbar_wait(&full[b], (uint32_t)(((c - c_lo) / STAGES) & 1), &abort_flag, dstatus);
        const WStage &S = st[b];
        const int t0 = ready ? warp * kWSlice : 0, t1 = ready ? t0 + kWSlice : 0;
        const uint32_t head = ready ? S.fix[warp] : 0u, tail = ready ? S.fix[kWWarps + warp] : 0u;
        const char *trow = reinterpret_cast<const char *>(&S.tile[lane][0]);
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, acc = 0.f;
        // the open run: the shared address of its histogram entry and its
        // sum so far, which starts from the entry's old value (a run inside
        // the slice: no other run of the block has its bin, so the entries a
        // batch reads at its start are ones no earlier run wrote; a run
        // crossing the slice's end: the warp's tail column, zero).  Before
        // the slice's first run start the open entry is the warp's head
        // column if the slice begins inside a run, else the spare column B.
        const uint32_t head_col = hbase + (uint32_t)(B + 1 + warp) * 4u;
        uint32_t cur = (head & kWCross) ? head_col : hbase + (uint32_t)B * 4u;
        // batches of eight positions: every load of a batch (tile values,
        // powers, the histogram entries of the runs it starts) is issued
        // before its arithmetic, and a run's close is a predicated store, not
        // a branch; a word carries its column's byte offset, its bin and
        // whether it starts one; the slice is a whole number of batches
        // (fillers read the zero column and start no run)
        for (int t = t0; t < t1; t += 8) {
            const uint4 ca = *reinterpret_cast<const uint4 *>(&S.pt[t]);
            const uint4 cb = *reinterpret_cast<const uint4 *>(&S.pt[t + 4]);
            const uint4 ba = *reinterpret_cast<const uint4 *>(&S.pt[kWBlock + t]);
            const uint4 bb = *reinterpret_cast<const uint4 *>(&S.pt[kWBlock + t + 4]);
            uint32_t cw[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
            uint32_t bw[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
#ifdef VUP_DEBUG
            // (debug build: a column past the tile reads the zero column; a
            // histogram entry past the row lands in the spare column)
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (!VUP_DBG_IN(cw[u] >> 2, kWBlock + 1, dstatus) || (cw[u] & 3u)) cw[u] = kWFillerCol;
                if ((bw[u] & 1u) && !VUP_DBG_IN((bw[u] - 1u) >> 2, ld, dstatus)) bw[u] = (uint32_t)B * 4u + 1u;
            }
#endif
            float wv[8], hv[8];
            uint32_t ha[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) wv[u] = *reinterpret_cast<const float *>(trow + cw[u]);
            // a run's first position: its entry's address is hbase + (bw - 1);
            // elsewhere ha and hv are not used
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                ha[u] = hbase_m1 + bw[u];
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p ld.shared.f32 %0, [%1];\n\t}"
                             : "=f"(hv[u])
                             : "r"(ha[u]), "r"(bw[u] & 1u));
            }
            // the batch's eight z in two broadcast loads; powers by repeated
            // multiplication in FP32, as the other forms take them
            const float4 za = *reinterpret_cast<const float4 *>(&S.z[t]);
            const float4 zb = *reinterpret_cast<const float4 *>(&S.z[t + 4]);
            const float zv[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float p1 = zv[u], p2 = p1 * p1, p3 = p2 * p1, p4 = p3 * p1;
                m0 = fmaf(wv[u], p1, m0);
                m1 = fmaf(wv[u], p2, m1);
                m2 = fmaf(wv[u], p3, m2);
                m3 = fmaf(wv[u], p4, m3);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t st_u = bw[u] & 1u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.shared.f32 [%0], %1;\n\t}"
                             ::"r"(cur), "f"(acc), "r"(st_u)
                             : "memory");
                acc = (st_u ? hv[u] : acc) + wv[u];
                cur = st_u ? ha[u] : cur;
            }
        }
        if (t0 < t1) {
            asm volatile("st.shared.f32 [%0], %1;" ::"r"(cur), "f"(acc) : "memory");
            // crossing runs: this slice's part, from the warp's own columns,
            // added to the bin atomically (other slices add their parts)
            float *hrow_w = H + lane * ld;
            if ((head & kWCross) && VUP_DBG_IN(head & 0x7fffu, B, dstatus))
                atomicAdd(hrow_w + (head & 0x7fffu), hrow_w[B + 1 + warp]);
            if (tail & kWCross) {
                if (VUP_DBG_IN(tail & 0x7fffu, B, dstatus))
                    atomicAdd(hrow_w + (tail & 0x7fffu), hrow_w[B + 1 + kWWarps + warp]);
                hrow_w[B + 1 + kWWarps + warp] = 0.f;
            }
        }
        two_sum_acc(mhi[0], mlo[0], m0);
        two_sum_acc(mhi[1], mlo[1], m1);
        two_sum_acc(mhi[2], mlo[2], m2);
        two_sum_acc(mhi[3], mlo[3], m3);
        // buffer b and the histogram rows are free again; every thread learns
        // at once whether any wait expired (so all warps stop issuing
        // together and every issued phase gets all its arrivals)
        stop = __syncthreads_or(ready ? 0 : 1) != 0 || stop;
    }
    if (stop) {
        // drain: wait (bounded) for the last phase staged into each buffer,
        // then leave without writing partial results
        if (threadIdx.x == 0)
            for (int64_t i = issued > STAGES ? issued - STAGES : 0; i < issued; ++i)
                mbar_drain(&full[i % STAGES], (uint32_t)((i / STAGES) & 1));
        return;
    }
    // the warps' moment sums of each row, reduced through the idle stage buffers
    double *red = reinterpret_cast<double *>(wsm);  // [warps][kWRows][4]
#pragma unroll
    for (int j = 0; j < 4; ++j) red[(warp * kWRows + lane) * 4 + j] = (double)mhi[j] + (double)mlo[j];
    __syncthreads();
    if (threadIdx.x < kWRows * 4) {
        const int r = threadIdx.x >> 2, j = threadIdx.x & 3;
        double v = 0.0;
        for (int q = 0; q < kWWarps; ++q) v += red[(q * kWRows + r) * 4 + j];
        if (k0 + r < K) mpart[(split * K + k0 + r) * 4 + j] = v;
    }
    for (int e = threadIdx.x; e < kWRows * B; e += blockDim.x) {
        const int r = e / B, bb = e - r * B;
        if (k0 + r < K) hpart[(split * K + k0 + r) * B + bb] = H[r * ld + bb];
    }
}

// Block sort of the grid points by bin (once per model): one CTA of 256
// threads per block sorts the keys bin << 8 | local index (bitonic, in
// shared memory) and writes, in sorted order, the column words, the
// histogram words (see WStage) and z = y / s_abs (FP32, as the other
// supplied-weights kernels form it), and for each warp slice the
// bins of the runs that cross its start and its end.  Positions past the
// grid's end sort last.
__global__ void __launch_bounds__(kWBlock) k_wsort_blocks(const int32_t *__restrict__ bins,
                                                          const double *__restrict__ y, int64_t N,
                                                          const double *__restrict__ scale, int B,
                                                          uint32_t *__restrict__ wpt, float *__restrict__ wz,
                                                          uint16_t *__restrict__ wfix) {
    __shared__ uint32_t key[kWBlock];
    const int t = threadIdx.x;
    const int64_t c = blockIdx.x, col0 = c * kWBlock;
    const int nv = (int)min((int64_t)kWBlock, N - col0);
    key[t] = t < nv ? ((uint32_t)bins[col0 + t] << 8) | (uint32_t)t : 0xffffffffu;
    __syncthreads();
    for (int size = 2; size <= kWBlock; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int o = t ^ stride;
            if (o > t) {
                const bool up = (t & size) == 0;
                const uint32_t a = key[t], bb = key[o];
                if ((a > bb) == up) {
                    key[t] = bb;
                    key[o] = a;
                }
            }
            __syncthreads();
        }
    auto bin_at = [&](int q) { return key[q] >> 8; };
    // position q continues the run of q - 1 (q a real position)
    auto cont = [&](int q) { return q > 0 && q < nv && bin_at(q) == bin_at(q - 1); };
    uint32_t cword = kWFillerCol, bword = 0u;
    float zp = 0.f;
    if (t < nv) {
        const uint32_t kw = key[t];
        const int w = t / kWSlice, next = (w + 1) * kWSlice;  // first position of the next slice
        cword = (kw & 0xffu) << 2;
        if (!cont(t)) {
            const bool crosses = next < nv && bin_at(next) == (kw >> 8);
            bword = ((crosses ? (uint32_t)(B + 1 + kWWarps + w) : (kw >> 8)) << 2) | 1u;
        }
        const float p = (float)(y[col0 + (kw & 0xffu)] / scale[kScaleAbs]);
        zp = p;
    }
    wpt[c * 2 * kWBlock + t] = cword;
    wpt[c * 2 * kWBlock + kWBlock + t] = bword;
    wz[c * kWBlock + t] = zp;
    if (t < kWWarps) {
        const int p0 = t * kWSlice, p1 = p0 + kWSlice;
        // head: the slice begins inside a run; tail: a run that starts in the
        // slice continues into the next one
        const bool head = cont(p0);
        const bool tail = cont(p1) && !(head && bin_at(p0) == bin_at(p1));
        wfix[c * kWFix + t] = head ? (uint16_t)(bin_at(p0) | kWCross) : 0;
        wfix[c * kWFix + kWWarps + t] = tail ? (uint16_t)(bin_at(p1) | kWCross) : 0;
    }
}

__global__ void k_weights_finish(const double *__restrict__ mpart, const float *__restrict__ hpart,
                                 int64_t n_split, int64_t K, int B, int J, const double *__restrict__ scale,
                                 double *__restrict__ raw, float *__restrict__ hist) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (hist && e < K * B) {
        // the splits' partial rows as an FP32 TwoSum pair (about 2^-44
        // relative to the sum of magnitudes) on the FP32 pipes: FP64 adds
        // run at a small fraction of the FP32 rate here
        float sh = 0.f, sl = 0.f;
#pragma unroll 4
        for (int64_t q = 0; q < n_split; ++q) two_sum_acc(sh, sl, hpart[q * K * B + e]);
        hist[e] = (float)((double)sh + (double)sl);
    }
    if (raw && e < K * J) {
        const int64_t k = e / J;
        const int j = (int)(e - k * J);
        double s = 0.0;
        for (int64_t q = 0; q < n_split; ++q) s += mpart[(q * K + k) * 4 + j];
        double sp = scale[kScaleAbs];
        for (int q = 0; q < j; ++q) sp *= scale[kScaleAbs];
        raw[e] = s * sp;
    }
}

__global__ void k_z32(const double *__restrict__ y, int64_t N, const double *__restrict__ scale,
                      float *__restrict__ z32) {
    const double s = scale[kScaleAbs];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        z32[i] = (float)(y[i] / s);
}

}  // namespace

static DevBuf g_wz32, g_wmpart, g_whpart;  // process-wide scratch of this path

vup_status vup_weights_path(vup_grid g, int64_t K, const float *W, double *raw, float *hist, cudaStream_t s) {
    const int64_t N = g->N;
    const int B = g->B;
    vup_status st;
    const bool aligned = N % 4 == 0 && (reinterpret_cast<uintptr_t>(W) & 15) == 0;
    // a forced form (vup_set_weights_form) where it applies, else the first
    // that does: the sorted walk, the row-per-lane form, the general one
    const int form = g->weights_form;
    if ((form == -1 || form == 0) && B <= 1024 && aligned && ceil_div64(K, kWRows) <= 65535) {
        const int64_t n_blk = ceil_div64(N, kWBlock);
        if (g->wsort_gen != g->model_gen) {
            if ((st = devbuf_reserve(g->wsort_pt, sizeof(uint32_t) * n_blk * 2 * kWBlock)) != VUP_OK ||
                (st = devbuf_reserve(g->wsort_z, sizeof(float) * n_blk * kWBlock)) != VUP_OK ||
                (st = devbuf_reserve(g->wsort_fix, sizeof(uint16_t) * kWFix * n_blk)) != VUP_OK)
                return st;
            k_wsort_blocks<<<(unsigned)n_blk, kWBlock, 0, s>>>(g->bins, g->y, N, g->ydev_scale, B,
                                                                (uint32_t *)g->wsort_pt.p, (float *)g->wsort_z.p,
                                                                (uint16_t *)g->wsort_fix.p);
            VUP_CHECK_LAUNCH();
            g->wsort_gen = g->model_gen;
        }
        const int64_t rows = ceil_div64(K, kWRows);
        // two CTAs of two stages per SM when their histogram rows fit (the
        // walks of two CTAs overlap each other's barriers; measured faster
        // than one CTA of four stages), else one CTA with as many stages as
        // shared memory holds, up to four
        const size_t hbytes = sizeof(float) * (size_t)kWRows * w_hist_ld(B);
        const size_t cap = 227 * 1024;
        const bool two_ctas = 2 * (sizeof(WStage) * 2 + hbytes) <= cap;
        int stages = two_ctas ? 2 : 4;
        while (stages > 2 && sizeof(WStage) * stages + hbytes > cap) --stages;
        const size_t smem = sizeof(WStage) * stages + hbytes;
        // column splits: each CTA over at most kWMaxBlocksPerCta blocks; among
        // the counts that allows, the one with the shortest schedule of
        // (waves of CTAs) x (blocks per CTA), searched up to 16 waves (past
        // that the last wave's tail costs little and the partial histograms
        // grow with the count)
        const int64_t slots = (int64_t)vup_num_sms() * (two_ctas ? 2 : 1);
        const int64_t lo_split = std::min<int64_t>(ceil_div64(n_blk, kWMaxBlocksPerCta), n_blk);
        const int64_t hi_split = std::max<int64_t>(lo_split, std::min<int64_t>(n_blk, 16 * slots / rows));
        int64_t n_split = lo_split, best = -1;
        for (int64_t q = lo_split; q <= hi_split; ++q) {
            const int64_t cost = ceil_div64(q * rows, slots) * ceil_div64(n_blk, q);
            if (best < 0 || cost < best) best = cost, n_split = q;
        }
        if ((st = devbuf_reserve(g_wmpart, sizeof(double) * 4 * K * n_split)) != VUP_OK) return st;
        if ((st = devbuf_reserve(g_whpart, sizeof(float) * (size_t)B * K * n_split)) != VUP_OK) return st;
        VUP_PROF("weights_stream", s, 2);
        dim3 grd((unsigned)n_split, (unsigned)rows);
        auto launch = [&](auto kern) -> vup_status {
            VUP_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<grd, kWThreads, smem, s>>>(W, K, N, (const uint32_t *)g->wsort_pt.p, (const float *)g->wsort_z.p,
                                             (const uint16_t *)g->wsort_fix.p, B, n_split, (double *)g_wmpart.p,
                                             (float *)g_whpart.p, g->dstatus);
            return VUP_OK;
        };
        if (two_ctas)
            st = launch(k_weights_sorted<2, 2>);
        else if (stages == 4)
            st = launch(k_weights_sorted<4, 1>);
        else if (stages == 3)
            st = launch(k_weights_sorted<3, 1>);
        else
            st = launch(k_weights_sorted<2, 1>);
        if (st != VUP_OK) return st;
        VUP_CHECK_LAUNCH();
        const int64_t tot = std::max<int64_t>(K * B, K * g->J);
        k_weights_finish<<<(unsigned)ceil_div64(tot, 256), 256, 0, s>>>((const double *)g_wmpart.p,
                                                                        (const float *)g_whpart.p, n_split, K, B,
                                                                        g->J, g->ydev_scale, raw, hist);
        VUP_CHECK_LAUNCH();
        return VUP_OK;
    }
    // the other forms read the FP32 powers z = y / s_abs in grid order
    if ((st = devbuf_reserve(g_wz32, sizeof(float) * (N + 4))) != VUP_OK) return st;
    k_z32<<<(unsigned)std::min<int64_t>(ceil_div64(N, 256), 4096), 256, 0, s>>>(g->y, N, g->ydev_scale,
                                                                                (float *)g_wz32.p);
    VUP_CHECK_LAUNCH();
    if (B <= 1024 && form != 2) {
        const int64_t rows = ceil_div64(K, kRowsT);
        int64_t n_split = std::max<int64_t>(1, (int64_t)vup_num_sms() * 4 / std::max<int64_t>(rows, 1));
        n_split = std::min<int64_t>(n_split, std::max<int64_t>(1, N / 8192));
        if ((st = devbuf_reserve(g_wmpart, sizeof(double) * 4 * K * n_split)) != VUP_OK) return st;
        if ((st = devbuf_reserve(g_whpart, sizeof(float) * (size_t)B * K * n_split)) != VUP_OK) return st;
        const size_t smem = sizeof(float) * (size_t)kRowsT * (B + 1);
        VUP_PROF("weights_stream", s, 3);
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_weights_t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_weights_t<<<dim3((unsigned)n_split, (unsigned)rows), kThreads, smem, s>>>(
            W, K, N, (const float *)g_wz32.p, g->bins, B, n_split, (double *)g_wmpart.p, (float *)g_whpart.p);
        VUP_CHECK_LAUNCH();
        const int64_t tot = std::max<int64_t>(K * B, K * g->J);
        k_weights_finish<<<(unsigned)ceil_div64(tot, 256), 256, 0, s>>>((const double *)g_wmpart.p,
                                                                        (const float *)g_whpart.p, n_split, K, B,
                                                                        g->J, g->ydev_scale, raw, hist);
        VUP_CHECK_LAUNCH();
        return VUP_OK;
    }
    const int RB = B <= 3072 ? 8 : (B <= 6144 ? 4 : 2);
    const int64_t rows = ceil_div64(K, RB);
    if (rows > 65535) return VUP_ERR_UNSUPPORTED;  // one CTA row per RB densities
    int64_t n_split = std::max<int64_t>(1, (int64_t)vup_num_sms() * 8 / std::max<int64_t>(rows, 1));
    n_split = std::min<int64_t>(n_split, std::max<int64_t>(1, N / 4096));
    if ((st = devbuf_reserve(g_wmpart, sizeof(double) * 4 * K * n_split)) != VUP_OK) return st;
    if ((st = devbuf_reserve(g_whpart, sizeof(float) * (size_t)B * K * n_split)) != VUP_OK) return st;
    const size_t smem = sizeof(float) * (size_t)RB * B;
    dim3 grd((unsigned)n_split, (unsigned)rows);
    VUP_PROF("weights_stream", s, 3);
    if (RB == 8) {
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_weights<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
        k_weights<8><<<grd, kThreads, smem, s>>>(W, K, N, (const float *)g_wz32.p, g->bins, B, n_split,
                                                 (double *)g_wmpart.p, (float *)g_whpart.p);
    } else if (RB == 4) {
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_weights<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
        k_weights<4><<<grd, kThreads, smem, s>>>(W, K, N, (const float *)g_wz32.p, g->bins, B, n_split,
                                                 (double *)g_wmpart.p, (float *)g_whpart.p);
    } else {
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_weights<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
        k_weights<2><<<grd, kThreads, smem, s>>>(W, K, N, (const float *)g_wz32.p, g->bins, B, n_split,
                                                 (double *)g_wmpart.p, (float *)g_whpart.p);
    }
    VUP_CHECK_LAUNCH();
    const int64_t tot = std::max<int64_t>(K * B, K * g->J);
    k_weights_finish<<<(unsigned)ceil_div64(tot, 256), 256, 0, s>>>((const double *)g_wmpart.p,
                                                                    (const float *)g_whpart.p, n_split, K, B,
                                                                    g->J, g->ydev_scale, raw, hist);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}
