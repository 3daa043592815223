// Moment contraction on the 5th-generation tensor cores (tcgen05 + TMEM).
//
//   T[k, (q, j)] = sum_r g_red(k, r) z_(q,r)^(j+1), z = (y - c) / s (GEMM, Eq. VUP
//   M[k, j]     += sum_q g_rest(k, q) T[k, (q, j)]               as moments)
//
// BF16x3: every FP32 operand is split into bf16 hi + lo and the product is
// formed as hi*hi + hi*lo + lo*hi with FP32 accumulation in TMEM (the lo*lo
// term, ~2^-16 relative, is dropped).  Operand tiles are staged by TMA
// (cp.async.bulk.tensor, 128-byte swizzle) into a 2-stage shared-memory ring;
// one thread issues tcgen05.mma; the accumulator is double-buffered in TMEM
// (2 x 256 columns) so that the epilogue of one tile overlaps the main loop
// of the next.  The epilogue reads TMEM with tcgen05.ld, multiplies by the
// rest-axis density factors generated from the factor tables, reduces over
// the tile's q values and writes FP32 partials that an FP64 kernel sums.
//
// Warp roles (192 threads): warp 0 = TMA producer, warp 1 = MMA issuer,
// warps 2..5 = epilogue (one TMEM lane quadrant each).  Persistent CTAs walk
// the (row tile, column tile) list with a static stride.  Every mbarrier wait
// is bounded; on expiry the kernel records VUP_DSTAT_TIMEOUT, drains what it
// issued and returns.
#include "vup_internal.cuh"
#include "vup_async.cuh"

#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <vector>

namespace {

constexpr int BM = 128, BN = 256, BK = 64;  // BK in BF16 elements: 128-byte rows
constexpr int BK_TF32 = 32;                     // TF32 operands: 32 x 4 bytes per row
constexpr int kSplitTerms = 1024;               // reduction terms per accumulator
constexpr int STAGES = 2;
constexpr int A_BYTES = BM * BK * 2;            // 16 KB per bf16 plane
constexpr int B_BYTES = BN * BK * 2;            // 32 KB per bf16 plane
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int TMEM_COLS = 512;                  // 2 accumulators of BN fp32 columns
constexpr int kThreads = 192;

using namespace vup_async;

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

// UMMA shared-memory descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row core groups 1024 bytes apart (SBO), version 1 (sm_100+).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3fff);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // descriptor version
    d |= (uint64_t)2 << 61;               // SWIZZLE_128B
    return d;
}

// Instruction descriptor: D = FP32, A and B K-major, M = 128, N = bn (a
// multiple of 16 up to 256); operand type BF16 (kind::f16) or TF32
// (kind::tf32).
template <int KIND>
__host__ __device__ constexpr uint32_t idesc_for(int bn) {
    return (1u << 4) | ((KIND ? 2u : 1u) << 7) | ((KIND ? 2u : 1u) << 10) | ((uint32_t)(bn >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accum) {
    if (KIND == 0)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
            : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcEpi {
    const float *g_rest0;      // [n_rest0][K_pad]
    const float *g_rest1;      // 3-D second rest axis or nullptr
    int64_t n_rest1;
    int64_t Q;                 // rest points
    const DensConst *dconst;   // IPSA weights (rest axis)
    int ndim, rest_axis;
};

// Batched instance descriptor (device memory, 128-byte aligned): the four
// operand tensor maps of one instance, its column-tile width bn (64, 128 or
// 256; the B maps' box is bn rows) and its epilogue parameters.
struct alignas(128) TcInst {
    CUtensorMap maps[4];  // A hi, A lo, B hi, B lo
    TcEpi ep;
    int64_t K_pad;
    float *part;
    int n_n, n_kb, bn;
};
struct TcTile {
    int32_t inst, m, n, pad;
};

// Work schedule of one (non-batched) contraction.  The tiles of a row tile
// (128 densities) and reduction split are grouped into items that one CTA
// processes in a row, summing their epilogue results in registers and
// writing one partial column per item.  Plain items are single column tiles.
// "Row-block" items (3-D grids whose second rest axis has a multiple of 64
// points): a 256-column tile covers 64 consecutive points of that axis for
// one index of the first, so an item takes L consecutive first-axis indices
// at one second-axis block; its epilogue loads the block's 64 factors of the
// second axis once and one factor of the first axis per tile.
struct TcSched {
    int n_m, n_n, n_split;  // row tiles, column tiles, reduction splits
    int split_terms;        // reduction terms per split (a multiple of 64)
    int per_row;            // items per (row tile, split) = partial columns per split
    int fast;               // row-block items
    int T1, L, n0;          // row-block: column tiles per first-axis index, indices per item, first-axis size
};
constexpr int kItemRows = 16;  // first-axis indices per row-block item

// kBatched == false: one instance, tensor maps as kernel parameters, items
// of the schedule S.  kBatched == true: items are single tiles from a work
// list over many instances and each tile's maps and epilogue parameters come
// from its instance descriptor.  KIND 0: BF16 operands (kind::f16, 64 per
// 128-byte row); KIND 1: TF32 operands (kind::tf32, 32 per row).  terms = 3:
// hi*hi + hi*lo + lo*hi; terms = 1: hi*hi only (the lo planes are not read).
template <int NOUT, bool kBatched, int KIND = 0>
__global__ void __launch_bounds__(kThreads, 1)
k_moments_tc(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
             const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, TcSched S,
             int n_kb, int64_t K_pad, TcEpi ep, float *__restrict__ part, const TcInst *__restrict__ insts,
             const TcTile *__restrict__ tiles, int n_tiles_batched, int *__restrict__ dstatus, int terms = 3) {
    pdl_trigger();
    pdl_wait();
    constexpr int BKE = KIND ? BK_TF32 : BK;  // operand elements per 128-byte row
    // split reduction: n_split accumulators of at most kSplitTerms terms each
    // (the tensor cores' FP32 accumulation error grows with the reduction
    // length); every split writes its own partial columns, summed by the
    // finish
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(drain + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = kBatched ? n_tiles_batched : S.n_m * S.n_split * S.per_row;
    // item -> (instance, row tile, split, item column, tile count)
    auto item_at = [&](int it, int &m, int &sp, int &ic, int &cnt, const TcInst *&in) {
        if (kBatched) {
            const TcTile tt = tiles[it];
            in = insts + tt.inst;
            m = tt.m;
            sp = 0;
            ic = tt.n;
            cnt = 1;
            return;
        }
        in = nullptr;
        const int per = S.n_split * S.per_row;
        m = it / per;
        const int r = it - m * per;
        sp = r / S.per_row;
        ic = r - sp * S.per_row;
        cnt = S.fast ? min(S.L, S.n0 - (ic / S.T1) * S.L) : 1;
    };
    // column tile of the i-th tile of item column ic
    auto tile_n = [&](int ic, int i) -> int {
        if (!kBatched && S.fast) return ((ic / S.T1) * S.L + i) * S.T1 + ic % S.T1;
        return ic;
    };
    // k-block range and tile width of a split
    auto kb_range = [&](int sp, const TcInst *in, int &kb0, int &kb1, int &bn) {
        if (kBatched) {
            kb0 = 0;
            kb1 = in->n_kb;
            bn = in->bn;
        } else {
            const int split_kb = S.split_terms / BKE;
            kb0 = sp * split_kb;
            kb1 = min(n_kb, kb0 + split_kb);
            bn = BN;
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            uint32_t it_s = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                int m, sp, ic, cnt, kb0, kb1, bn;
                const TcInst *in;
                item_at(it, m, sp, ic, cnt, in);
                kb_range(sp, in, kb0, kb1, bn);
                const CUtensorMap *mAh = kBatched ? &in->maps[0] : &tmAh;
                const CUtensorMap *mAl = kBatched ? &in->maps[1] : &tmAl;
                const CUtensorMap *mBh = kBatched ? &in->maps[2] : &tmBh;
                const CUtensorMap *mBl = kBatched ? &in->maps[3] : &tmBl;
                for (int i = 0; i < cnt && ok; ++i) {
                    const int n = tile_n(ic, i);
                    for (int kb = kb0; kb < kb1; ++kb, ++it_s) {
                        const int s = it_s % STAGES;
                        if (!mbar_wait(&empty[s], ((it_s / STAGES) & 1) ^ 1, abort_flag, dstatus)) {
                            ok = false;
                            break;
                        }
                        uint8_t *st = smem + s * STAGE_BYTES;
                        mbar_expect_tx(&full[s], (terms == 3 ? 2 : 1) * (A_BYTES + 128 * bn));
                        tma_load_2d(st, mAh, &full[s], kb * BKE, m * BM);
                        tma_load_2d(st + 2 * A_BYTES, mBh, &full[s], kb * BKE, n * bn);
                        if (terms == 3) {
                            tma_load_2d(st + A_BYTES, mAl, &full[s], kb * BKE, m * BM);
                            tma_load_2d(st + 2 * A_BYTES + B_BYTES, mBl, &full[s], kb * BKE, n * bn);
                        }
                    }
                }
            }
            // drain: every issued stage must land before shared memory is released
            if (!ok) {
                for (uint32_t j = (it_s > (uint32_t)STAGES ? it_s - STAGES : 0); j < it_s; ++j) {
                    for (uint32_t i = 0; i < kSpinLimit && !mbar_try_wait(&full[j % STAGES], (j / STAGES) & 1); ++i) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t it_s = 0, tile_it = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                int m_, sp, ic, cnt, kb0, kb1, bn;
                const TcInst *in_;
                item_at(it, m_, sp, ic, cnt, in_);
                kb_range(sp, in_, kb0, kb1, bn);
                const uint32_t idesc = idesc_for<KIND>(bn);
                for (int i = 0; i < cnt; ++i, ++tile_it) {
                    const int b = tile_it & 1;
                    if (!mbar_wait(&tempty[b], ((tile_it >> 1) & 1) ^ 1, abort_flag, dstatus)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dcol = tmem_base + (uint32_t)(b * BN);
                    for (int kb = kb0; kb < kb1; ++kb, ++it_s) {
                        const int s = it_s % STAGES;
                        if (!mbar_wait(&full[s], (it_s / STAGES) & 1, abort_flag, dstatus)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a_hi = smem_u32(smem + s * STAGE_BYTES);
                        const uint32_t a_lo = a_hi + A_BYTES;
                        const uint32_t b_hi = a_hi + 2 * A_BYTES;
                        const uint32_t b_lo = b_hi + B_BYTES;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            // 32 bytes along K inside the swizzle atom: 16 BF16 or 8 TF32
                            const uint32_t off = kk * 32;
                            const uint32_t acc0 = (kb > kb0 || kk > 0) ? 1u : 0u;
                            if (terms == 3) {
                                umma<KIND>(dcol, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc, acc0);
                                umma<KIND>(dcol, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc, 1u);
                                umma<KIND>(dcol, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, 1u);
                            } else {
                                umma<KIND>(dcol, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, acc0);
                            }
                        }
                        umma_commit(&empty[s]);
                    }
                    if (!ok) break;
                    umma_commit(&tfull[b]);
                }
            }
            // all MMAs issued by this thread complete before TMEM is released
            umma_commit(drain);
            for (uint32_t i = 0; i < kSpinLimit && !mbar_try_wait(drain, 0); ++i) {
            }
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        uint32_t tile_it = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
            int m, sp, ic, cnt, kb0, kb1, bn;
            const TcInst *in;
            item_at(it, m, sp, ic, cnt, in);
            kb_range(sp, in, kb0, kb1, bn);
            const TcEpi &E = kBatched ? in->ep : ep;
            const int64_t Kp = kBatched ? in->K_pad : K_pad;
            const int ncols = kBatched ? in->n_n : S.n_split * S.per_row;  // partial columns
            const int col = kBatched ? ic : sp * S.per_row + ic;
            float *const P = kBatched ? in->part : part;
            const int64_t k = (int64_t)m * BM + row;
            float out[NOUT][4];
#pragma unroll
            for (int o = 0; o < NOUT; ++o)
#pragma unroll
                for (int j = 0; j < 4; ++j) out[o][j] = 0.f;
            DensConst dc{};
            if (NOUT == 3) dc = E.dconst[k * E.ndim + E.rest_axis];
            const bool rows_fast = NOUT == 1 && !kBatched && S.fast;
            // row-block item: the 64 second-axis factors of its block, loaded once
            float g1v[64];
            if (rows_fast) {
                const float *g1 = E.g_rest1 + (int64_t)(ic % S.T1) * 64 * Kp + k;
#pragma unroll
                for (int e = 0; e < 64; ++e) g1v[e] = g1[e * Kp];
            }
            for (int i = 0; i < cnt; ++i, ++tile_it) {
                const int n = tile_n(ic, i);
                float g0 = 0.f;
                if (rows_fast) g0 = E.g_rest0[(int64_t)((ic / S.T1) * S.L + i) * Kp + k];
                const int b = tile_it & 1;
                if (!mbar_wait(&tfull[b], (tile_it >> 1) & 1, abort_flag, dstatus)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tbase = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * BN);
                if (rows_fast) {
#pragma unroll
                    for (int ch = 0; ch < BN / 32; ++ch) {
                        float v[32];
                        tmem_ld32(tbase + ch * 32, v);
#pragma unroll
                        for (int qq = 0; qq < 8; ++qq) {
                            const float w = g0 * g1v[ch * 8 + qq];
#pragma unroll
                            for (int j = 0; j < 4; ++j) out[0][j] = fmaf(w, v[qq * 4 + j], out[0][j]);
                        }
                    }
                } else {
#pragma unroll 1
                    for (int ch = 0; ch < bn / 32; ++ch) {
                        float v[32];
                        tmem_ld32(tbase + ch * 32, v);
                        const int64_t q0 = (int64_t)n * (bn / 4) + ch * 8;
                        float e[8];
#pragma unroll
                        for (int qq = 0; qq < 8; ++qq) {
                            const int64_t q = q0 + qq;
                            float w = 0.f;
                            if (q < E.Q) {
                                if (E.g_rest1) {
                                    const int64_t qa = q / E.n_rest1, qb = q - qa * E.n_rest1;
                                    w = E.g_rest0[qa * Kp + k] * E.g_rest1[qb * Kp + k];
                                } else {
                                    w = E.g_rest0[q * Kp + k];
                                }
                            }
                            e[qq] = w;
                        }
#pragma unroll
                        for (int qq = 0; qq < 8; ++qq) {
                            float w[NOUT];
                            w[0] = e[qq];
                            if (NOUT == 3) {
                                const float tt = (float)(q0 + qq - dc.n) - dc.f;
                                const float u = tt * dc.r;
                                w[NOUT == 3 ? 1 : 0] = e[qq] * u;
                                w[NOUT == 3 ? 2 : 0] = e[qq] * u * u;
                            }
#pragma unroll
                            for (int o = 0; o < NOUT; ++o)
#pragma unroll
                                for (int j = 0; j < 4; ++j) out[o][j] = fmaf(w[o], v[qq * 4 + j], out[o][j]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[b]);
            }
            if (!ok) break;
#pragma unroll
            for (int o = 0; o < NOUT; ++o)
                *reinterpret_cast<float4 *>(P + (((int64_t)o * ncols + col) * Kp + k) * 4) =
                    make_float4(out[o][0], out[o][1], out[o][2], out[o][3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

// ---- host side: tensor maps -------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2-D map over a row-major [rows][ld] array of BF16 (box [box_rows][64])
// or, with f32, of TF32-in-float values (box [box_rows][32]): 128-byte rows.
bool make_map(CUtensorMap *m, const void *base, int64_t ld, int64_t rows, int box_rows, bool f32 = false) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * (f32 ? 4 : 2))};
    cuuint32_t box[2] = {(cuuint32_t)(f32 ? BK_TF32 : BK), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

// Schedule of a contraction over K_pad rows (see TcSched); its partial
// columns per row are n_split * per_row.  Splits of at most kSplitTerms
// terms; a reduction of one split of at least 2 * kMinSplitTerms terms is
// cut in two when that fills the persistent grid's last wave better (c2:
// 2048 items are 13.5 waves of 152 CTAs, 4096 half items 26.9), the
// epilogue of a half item being far shorter than its MMAs.
constexpr int kMinSplitTerms = 512;
static int tc_splits(const Orient &o) { return (int)ceil_div64(o.R_pad, kSplitTerms); }
static bool tc_can_halve(const Orient &o) { return tc_splits(o) == 1 && o.R_pad >= 2 * kMinSplitTerms; }
static TcSched tc_sched(const Orient &o, int64_t K_pad) {
    TcSched S{};
    S.n_m = (int)(K_pad / BM);
    S.n_n = (int)ceil_div64(o.NC, BN);
    S.n_split = tc_splits(o);
    S.split_terms = kSplitTerms;
    S.fast = o.n_rest_axes == 2 && o.rest_n[1] % (BN / 4) == 0;
    if (S.fast) {
        S.T1 = (int)(o.rest_n[1] / (BN / 4));
        S.n0 = (int)o.rest_n[0];
        S.L = kItemRows;
        S.per_row = S.T1 * (int)ceil_div64(S.n0, S.L);
    } else {
        S.T1 = 1;
        S.L = 1;
        S.n0 = S.n_n;
        S.per_row = S.n_n;
    }
    if (tc_can_halve(o)) {
        const int64_t sms = vup_num_sms(), items = (int64_t)S.n_m * S.per_row;
        auto fill = [&](int64_t it) { return (double)it / (double)(ceil_div64(it, sms) * sms); };
        if (fill(2 * items) > fill(items) + 0.02) {
            S.n_split = 2;
            S.split_terms = (int)(ceil_div64(o.R_pad, 2 * 64) * 64);
        }
    }
    return S;
}
int64_t vup_tc_col_tiles(const Orient &o, int64_t K) {
    const TcSched S = tc_sched(o, ceil_div64(K, 128) * 128);
    return (int64_t)S.n_split * S.per_row;
}
int64_t vup_tc_col_tiles_max(const Orient &o) {
    const TcSched S = tc_sched(o, BM);
    return (int64_t)S.n_split * S.per_row * (tc_can_halve(o) ? 2 : 1);
}

vup_status vup_moments_tc(vup_grid g, int64_t K, int orient, int n_out, float *part, cudaStream_t s, int kind,
                          int terms) {
    const Orient &o = g->orient[orient];
    const int64_t K_pad = ceil_div64(K, 128) * 128;
    const int64_t rows_b = ceil_div64(o.NC, 256) * 256;
    const bool f32 = kind == 1;
    const size_t esz = f32 ? 4 : 2;
    const char *ah = (const char *)(f32 ? g->atf_hi.p : g->atab_hi.p);
    const char *al = (const char *)(f32 ? g->atf_lo.p : g->atab_lo.p);
    if (orient == 1) {
        const size_t o0 = (size_t)K_pad * g->orient[0].R_pad * esz;
        ah += o0;
        al += o0;
    }
    const void *bh = f32 ? (const void *)g->ztf_hi[orient] : (const void *)g->zt_hi[orient];
    const void *bl = f32 ? (const void *)g->ztf_lo[orient] : (const void *)g->zt_lo[orient];
    CUtensorMap mAh, mAl, mBh, mBl;
    if (!make_map(&mAh, ah, o.R_pad, K_pad, BM, f32) || !make_map(&mAl, al, o.R_pad, K_pad, BM, f32) ||
        !make_map(&mBh, bh, o.R_pad, rows_b, BN, f32) || !make_map(&mBl, bl, o.R_pad, rows_b, BN, f32))
        return VUP_ERR_CUDA;
    TcEpi ep{};
    auto tab = [&](int axis) {
        int64_t off = 0;
        for (int q = 0; q < axis; ++q) off += g->n[q] * K_pad;
        return (const float *)g->ftab.p + off;
    };
    ep.g_rest0 = tab(o.rest_axes[0]);
    ep.g_rest1 = o.n_rest_axes > 1 ? tab(o.rest_axes[1]) : nullptr;
    ep.n_rest1 = o.n_rest_axes > 1 ? g->n[o.rest_axes[1]] : 1;
    ep.Q = o.Q;
    ep.dconst = (const DensConst *)g->dconst.p;
    ep.ndim = g->ndim;
    ep.rest_axis = o.rest_axes[0];
    const TcSched S = tc_sched(o, K_pad);
    const int n_kb = (int)(o.R_pad / (f32 ? BK_TF32 : BK));
    const int n_items = S.n_m * S.n_split * S.per_row;
    const int grid = std::min(n_items, vup_num_sms());
    const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
    if (f32) {
        if (n_out != 1) return VUP_ERR_UNSUPPORTED;
        VUP_PROF(terms == 3 ? "moments_tf32x3_tc" : "moments_tf32_tc", s, 1);
        VUP_CHECK_CUDA(
            cudaFuncSetAttribute(k_moments_tc<1, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_moments_tc<1, false, 1><<<grid, kThreads, smem, s>>>(mAh, mAl, mBh, mBl, S, n_kb, K_pad, ep, part,
                                                               nullptr, nullptr, 0, g->dstatus, terms);
        VUP_CHECK_LAUNCH();
        return VUP_OK;
    }
    VUP_PROF(n_out == 1 ? "moments_bf16x3_tc" : "ipsa_bf16x3_tc", s, 1);
    if (n_out == 1) {
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_moments_tc<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        VUP_CHECK_CUDA(launch_pdl(k_moments_tc<1, false>, dim3(grid), dim3(kThreads), smem, s, mAh, mAl, mBh, mBl, S,
                                  n_kb, K_pad, ep, part, (const TcInst *)nullptr, (const TcTile *)nullptr, 0,
                                  g->dstatus, 3));
    } else {
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_moments_tc<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_moments_tc<3, false><<<grid, kThreads, smem, s>>>(mAh, mAl, mBh, mBl, S, n_kb, K_pad, ep, part, nullptr,
                                                            nullptr, 0, g->dstatus, 3);
    }
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}

// Column tiles of an orientation at tile width bn.
int64_t vup_tc_col_tiles_bn(const Orient &o, int bn) { return ceil_div64(o.NC, bn); }

// Tile width of one instance: the smallest of 64 / 128 / 256 that covers the
// instance's columns, capped at bn_cap (narrower tiles waste less padding on
// small instances and give the persistent kernel finer work to balance).
int vup_tc_bn_for(const Orient &o, int bn_cap) {
    int bn = 64;
    while (bn < BN && bn < bn_cap && bn < o.NC) bn *= 2;
    return bn;
}

// Batched raw-moment contraction over n 2-D instances: instance i writes its
// partials [n_n][K_pad][4] to parts[i].  The tile list holds every instance's
// (row tile, column tile) pairs, longest reductions first.
struct TcPlan {
    DevBuf insts, tiles;
    int n_tiles = 0;
};

vup_status vup_tc_plan(int n, const vup_grid *gs, const int64_t *Ks, const int *bns, float *const *parts,
                       void **out) {
    std::vector<TcInst> insts(n);
    std::vector<std::pair<int64_t, TcTile>> work;
    for (int i = 0; i < n; ++i) {
        vup_grid g = gs[i];
        const Orient &o = g->orient[0];
        const int bn = bns[i];
        const int64_t K_pad = ceil_div64(Ks[i], 128) * 128;
        const int64_t rows_b = ceil_div64(o.NC, 256) * 256;
        TcInst &I = insts[i];
        memset(&I, 0, sizeof(I));
        if (!make_map(&I.maps[0], g->atab_hi.p, o.R_pad, K_pad, BM) ||
            !make_map(&I.maps[1], g->atab_lo.p, o.R_pad, K_pad, BM) ||
            !make_map(&I.maps[2], g->zt_hi[0], o.R_pad, rows_b, bn) ||
            !make_map(&I.maps[3], g->zt_lo[0], o.R_pad, rows_b, bn))
            return VUP_ERR_CUDA;
        auto tab = [&](int axis) {
            int64_t off = 0;
            for (int q = 0; q < axis; ++q) off += g->n[q] * K_pad;
            return (const float *)g->ftab.p + off;
        };
        I.ep.g_rest0 = tab(o.rest_axes[0]);
        I.ep.g_rest1 = nullptr;
        I.ep.n_rest1 = 1;
        I.ep.Q = o.Q;
        I.ep.dconst = (const DensConst *)g->dconst.p;
        I.ep.ndim = g->ndim;
        I.ep.rest_axis = o.rest_axes[0];
        I.K_pad = K_pad;
        I.part = parts[i];
        I.n_n = (int)vup_tc_col_tiles_bn(o, bn);
        I.n_kb = (int)(o.R_pad / BK);
        I.bn = bn;
        const int64_t cost = (int64_t)(I.n_kb + 2) * bn;
        for (int m = 0; m < (int)(K_pad / BM); ++m)
            for (int c = 0; c < I.n_n; ++c) work.push_back({cost, TcTile{i, m, c, 0}});
    }
    std::stable_sort(work.begin(), work.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::vector<TcTile> tiles(work.size());
    for (size_t q = 0; q < work.size(); ++q) tiles[q] = work[q].second;
    TcPlan *P = new TcPlan();
    P->n_tiles = (int)tiles.size();
    vup_status st;
    if ((st = devbuf_reserve(P->insts, sizeof(TcInst) * n)) != VUP_OK ||
        (st = devbuf_reserve(P->tiles, sizeof(TcTile) * std::max<size_t>(1, tiles.size()))) != VUP_OK) {
        devbuf_free(P->insts);
        devbuf_free(P->tiles);
        delete P;
        return st;
    }
    VUP_CHECK_CUDA(cudaMemcpy(P->insts.p, insts.data(), sizeof(TcInst) * n, cudaMemcpyHostToDevice));
    VUP_CHECK_CUDA(cudaMemcpy(P->tiles.p, tiles.data(), sizeof(TcTile) * tiles.size(), cudaMemcpyHostToDevice));
    const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
    VUP_CHECK_CUDA(cudaFuncSetAttribute(k_moments_tc<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    *out = P;
    return VUP_OK;
}

void vup_tc_plan_free(void *plan) {
    TcPlan *P = (TcPlan *)plan;
    if (!P) return;
    devbuf_free(P->insts);
    devbuf_free(P->tiles);
    delete P;
}

vup_status vup_tc_batched(void *plan, int *dstatus, cudaStream_t s) {
    const TcPlan *P = (const TcPlan *)plan;
    if (P->n_tiles == 0) return VUP_OK;
    const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
    const int grid = std::min(P->n_tiles, vup_num_sms());
    VUP_PROF("moments_bf16x3_tc_batched", s, 1);
    CUtensorMap dummy;
    memset(&dummy, 0, sizeof(dummy));
    TcEpi ep{};
    k_moments_tc<1, true><<<grid, kThreads, smem, s>>>(dummy, dummy, dummy, dummy, TcSched{}, 0, 0, ep, nullptr,
                                                       (const TcInst *)P->insts.p, (const TcTile *)P->tiles.p,
                                                       P->n_tiles, dstatus);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}
