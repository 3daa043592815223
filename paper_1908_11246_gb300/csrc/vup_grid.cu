// Grid-side steps of the VUP hot path, run once per (grid, model):
//   midpoint coordinates and model evaluation in FP64 (Sec. 2 model function,
//   Sec. 3 composite midpoint rule), the exact output range, per-point bin ids
//   (Eq. 4), a stable counting sort of the grid points by bin -- the CSR form
//   of the one-hot model matrix of Eq. MUP -- the run/chunk structure the
//   segmented histogram kernel walks, and the power tables ((y - c)/s)^j.
#include "vup_internal.cuh"

#include <math.h>

#include <algorithm>
#include <memory>

namespace {

constexpr int kSortTile = 2048;      // points per warp in the counting sort
constexpr int kSortWarps = 4;        // warps per CTA in the counting sort
// Packed sorted-point word: the gathered-axis row inside its part << 9 (the
// byte offset of its row in a 128-float shared-memory tile), run-end flag
// (bit 30), key-end flag (bit 31).
constexpr int kRowShift = 9;   // shared-memory tile rows of 512 bytes (128 floats)
constexpr int kRowBits = 9;    // row field width (tile rows < 512)
constexpr uint32_t kRunEnd = 1u << 30;
constexpr uint32_t kBinEnd = 1u << 31;

struct Theta {
    double t[8];
};

// Midpoint x_a = lo + (a + 1/2) h, with the product and sum rounded once each
// (no fused multiply-add), exactly as the FP64 oracle computes it.
__device__ __forceinline__ double grid_x(double lo, double h, int64_t a) {
    double t = (double)a + 0.5;
    return __dadd_rn(lo, __dmul_rn(t, h));
}

__device__ __forceinline__ double model_value(int model, const Theta &th, const double *x, int ndim) {
    switch (model) {
    case VUP_MODEL_SIN_QUAD_1D: {
        double s = sin(x[0]);
        double q = __dmul_rn(x[0], x[0]);
        return __dadd_rn(__dmul_rn(th.t[0], s), __dmul_rn(th.t[1], q));
    }
    case VUP_MODEL_SIN_SIN2_2D: {
        double s1 = sin(x[0]);
        double s2 = sin(x[1]);
        double q = __dmul_rn(s2, s2);
        return __dadd_rn(__dmul_rn(th.t[0], s1), __dmul_rn(th.t[1], q));
    }
    case VUP_MODEL_MIXED_3D: {
        double s1 = sin(x[0]);
        double s2 = sin(x[1]);
        double q = __dmul_rn(s2, s2);
        double x2 = __dmul_rn(x[2], x[2]);
        double x4 = __dmul_rn(x2, x2);
        double b = __dmul_rn(th.t[0], q);
        double c = __dmul_rn(th.t[1], x4);
        double c2 = __dmul_rn(c, s1);
        double r = __dadd_rn(s1, b);
        return __dadd_rn(r, c2);
    }
    case VUP_MODEL_OSCILLATOR_2D: {
        double w = x[0], z = x[1], T = th.t[0];
        double zw = __dmul_rn(z, w);
        double e = exp(-__dmul_rn(zw, T));
        double om = __dsub_rn(1.0, __dmul_rn(z, z));
        double wd = __dmul_rn(w, sqrt(om));
        double c = cos(__dmul_rn(wd, T));
        return __dmul_rn(e, c);
    }
    case VUP_MODEL_IPSA_EXAMPLE_2D: {
        double q = __dmul_rn(x[0], x[0]);
        double t = __dmul_rn(3.0, x[0]);
        double s = __dmul_rn(5.0, sin(t));
        double r = __dadd_rn(q, s);
        return __dadd_rn(r, x[1]);
    }
    case VUP_MODEL_POLY: {
        double r = th.t[0];
        for (int d = 0; d < ndim; ++d) {
            double a = __dmul_rn(th.t[1 + 2 * d], x[d]);
            double q = __dmul_rn(x[d], x[d]);
            double b = __dmul_rn(th.t[2 + 2 * d], q);
            r = __dadd_rn(r, a);
            r = __dadd_rn(r, b);
        }
        return r;
    }
    default:
        return __longlong_as_double(0x7ff8000000000000ll);
    }
}

struct GridGeom {
    int ndim;
    int64_t n[3];
    double lo[3];
    double h[3];
};

// Order-preserving map of a double to an unsigned key (for exact atomic min/max).
__device__ __forceinline__ unsigned long long dkey(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
    unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)u);
}

// Exact min / max of y into ext[0], ext[1] (order-preserving keys): reduced
// over the block first, then one atomic pair per block.  Called by every
// thread of the block (blockDim.x <= 1024).
__device__ __forceinline__ void range_reduce(unsigned long long mn, unsigned long long mx, unsigned long long *ext) {
    __shared__ unsigned long long s_mn[32], s_mx[32];
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn, o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, mx, o);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        s_mn[warp] = mn;
        s_mx[warp] = mx;
    }
    __syncthreads();
    if (warp == 0) {
        mn = lane < nw ? s_mn[lane] : ~0ull;
        mx = lane < nw ? s_mx[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn, o);
            const unsigned long long b = __shfl_xor_sync(0xffffffffu, mx, o);
            mn = a < mn ? a : mn;
            mx = b > mx ? b : mx;
        }
        if (lane == 0) {
            atomicMin(&ext[0], mn);
            atomicMax(&ext[1], mx);
        }
    }
}

// y at every grid point, and its exact range into ext (reset beforehand).
__global__ void k_model_eval(double *__restrict__ y, int64_t N, GridGeom G, int model, Theta th,
                             unsigned long long *ext) {
    pdl_trigger();
    pdl_wait();
    unsigned long long mn = ~0ull, mx = 0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = i;
        double x[3];
        for (int d = G.ndim - 1; d >= 0; --d) {
            int64_t a = rem % G.n[d];
            rem /= G.n[d];
            x[d] = grid_x(G.lo[d], G.h[d], a);
        }
        const double v = model_value(model, th, x, G.ndim);
        y[i] = v;
        const unsigned long long k = dkey(v);
        mn = k < mn ? k : mn;
        mx = k > mx ? k : mx;
    }
    range_reduce(mn, mx, ext);
}

// Separable built-in models: the transcendental and per-axis products are
// evaluated once per axis index (two FP64 terms per index, stored after the
// previous axes' terms), and every grid point only adds and multiplies its
// axes' terms -- the same operations in the same order as model_value, so y
// is bit-identical to the per-point evaluation.
__host__ __device__ inline bool model_separable(int model, int ndim) {
    return (model == VUP_MODEL_SIN_SIN2_2D && ndim == 2) || (model == VUP_MODEL_MIXED_3D && ndim == 3) ||
           (model == VUP_MODEL_IPSA_EXAMPLE_2D && ndim == 2) || (model == VUP_MODEL_POLY && ndim >= 2);
}

__global__ void k_axis_terms(GridGeom G, int model, Theta th, double2 *__restrict__ terms) {
    pdl_trigger();
    pdl_wait();
    int64_t off = 0;
    for (int d = 0; d < G.ndim; ++d) {
        for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < G.n[d];
             a += (int64_t)gridDim.x * blockDim.x) {
            const double x = grid_x(G.lo[d], G.h[d], a);
            double2 t = make_double2(0.0, 0.0);
            switch (model) {
            case VUP_MODEL_SIN_SIN2_2D:
                if (d == 0) {
                    t.x = __dmul_rn(th.t[0], sin(x));
                } else {
                    const double s2 = sin(x);
                    t.x = __dmul_rn(th.t[1], __dmul_rn(s2, s2));
                }
                break;
            case VUP_MODEL_MIXED_3D:
                if (d == 0) {
                    t.x = sin(x);
                } else if (d == 1) {
                    const double s2 = sin(x);
                    t.x = __dmul_rn(th.t[0], __dmul_rn(s2, s2));
                } else {
                    const double x2 = __dmul_rn(x, x);
                    t.x = __dmul_rn(th.t[1], __dmul_rn(x2, x2));
                }
                break;
            case VUP_MODEL_IPSA_EXAMPLE_2D:
                if (d == 0) t.x = __dadd_rn(__dmul_rn(x, x), __dmul_rn(5.0, sin(__dmul_rn(3.0, x))));
                else t.x = x;
                break;
            default:  // VUP_MODEL_POLY
                t.x = __dmul_rn(th.t[1 + 2 * d], x);
                t.y = __dmul_rn(th.t[2 + 2 * d], __dmul_rn(x, x));
                break;
            }
            terms[off + a] = t;
        }
        off += G.n[d];
    }
}

// Axis indices of a grid-stride walk over the flat index: decomposed once,
// then advanced by the stride's own decomposition with carries (no division
// per point).
struct IndexWalk {
    int32_t a[3], d[3], n[3];
    int ndim;
    __device__ __forceinline__ IndexWalk(const GridGeom &G, int64_t i0, int64_t step) : ndim(G.ndim) {
        int64_t r = i0, t = step;
        for (int q = 2; q >= 0; --q) {
            const int64_t nq = q < ndim ? G.n[q] : 1;
            n[q] = (int32_t)nq;
            a[q] = (int32_t)(r % nq);
            d[q] = (int32_t)(t % nq);
            r /= nq;
            t /= nq;
        }
        // the leading axis takes the rest of the stride without wrapping
        if (ndim >= 1) d[0] += (int32_t)(t * (int64_t)n[0]);
    }
    __device__ __forceinline__ void next() {
        int32_t c = 0;
        for (int q = 2; q >= 1; --q) {
            if (q >= ndim) continue;
            int32_t v = a[q] + d[q] + c;
            c = v >= n[q] ? 1 : 0;
            a[q] = c ? v - n[q] : v;
        }
        a[0] += d[0] + c;
    }
};

// y at axis indices a of a separable built-in model from its per-axis terms
// (bit-identical to the per-point evaluation).
__device__ __forceinline__ double combine_terms(const int32_t *a, const GridGeom &G, int model, const Theta &th,
                                                const double2 *__restrict__ terms) {
    const int64_t o1 = G.n[0], o2 = G.n[0] + G.n[1];
    double v;
    switch (model) {
    case VUP_MODEL_SIN_SIN2_2D:
    case VUP_MODEL_IPSA_EXAMPLE_2D:
        v = __dadd_rn(terms[a[0]].x, terms[o1 + a[1]].x);
        break;
    case VUP_MODEL_MIXED_3D: {
        const double s1 = terms[a[0]].x, b = terms[o1 + a[1]].x, c = terms[o2 + a[2]].x;
        v = __dadd_rn(__dadd_rn(s1, b), __dmul_rn(c, s1));
        break;
    }
    default: {  // VUP_MODEL_POLY
        v = th.t[0];
        int64_t off = 0;
        for (int d = 0; d < G.ndim; ++d) {
            const double2 t = terms[off + a[d]];
            v = __dadd_rn(v, t.x);
            v = __dadd_rn(v, t.y);
            off += G.n[d];
        }
        break;
    }
    }
    return v;
}

__global__ void k_model_combine(double *__restrict__ y, int64_t N, GridGeom G, int model, Theta th,
                                const double2 *__restrict__ terms, unsigned long long *ext) {
    pdl_trigger();
    pdl_wait();
    unsigned long long mn = ~0ull, mx = 0ull;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, step = (int64_t)gridDim.x * blockDim.x;
    IndexWalk w(G, i0, step);
    for (int64_t i = i0; i < N; i += step, w.next()) {
        const double v = combine_terms(w.a, G, model, th, terms);
        y[i] = v;
        const unsigned long long kv = dkey(v);
        mn = kv < mn ? kv : mn;
        mx = kv > mx ? kv : mx;
    }
    range_reduce(mn, mx, ext);
}

// Exact range of caller-supplied outputs (the model kernels reduce it as they write y).
__global__ void k_minmax(const double *__restrict__ y, int64_t N, unsigned long long *ext) {
    unsigned long long mn = ~0ull, mx = 0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long k = dkey(y[i]);
        mn = k < mn ? k : mn;
        mx = k > mx ? k : mx;
    }
    range_reduce(mn, mx, ext);
}

// Output range, and the power tables' reference point and scales {s, c,
// s_abs} (power_ref) written to s_out[0..2].
__device__ __forceinline__ void read_range(const unsigned long long *ext, double &ymin, double &ymax) {
    ymin = dkey_inv(ext[0]);
    ymax = dkey_inv(ext[1]);
}

__device__ __forceinline__ void write_scale(double ymin, double ymax, int64_t N, double *s_out) {
    double c, s, sa;
    power_ref(ymin, ymax, c, s, sa);
    s_out[kScaleS] = s;
    s_out[kScaleC] = c;
    s_out[kScaleAbs] = sa;
    s_out[kScaleP] = power_factor(N);
}

__global__ void k_scale(const unsigned long long *ext, int64_t N, double *s_out) {
    double ymin, ymax;
    read_range(ext, ymin, ymax);
    write_scale(ymin, ymax, N, s_out);
}

// Eq. 4 bin of one output value: t = (y - ymin) / (ymax - ymin), bin =
// min(floor(t B), B - 1), every operation correctly rounded and unfused, as
// in the FP64 oracle.  FP32 screen: t32 = (y - ymin) B / range lies within
// eps of the exact t; where no integer lies within eps of t32, floor(t32) is
// the bin, otherwise the FP64 expression decides (about one point in 10^4 on
// smooth models).  Error of t32: the FP32 roundings of y, ymin, the
// difference, B / range and the product, each <= 2^-24 relative: |t32 - t| <=
// 2^-24 ((|y| + |ymin|) B / range (2 + 2) + |t| 2); eps doubles that bound.
struct BinRule {
    double ymin, ymax, range;
    float ymin32, sc32;
    int B;
    __device__ __forceinline__ BinRule(const unsigned long long *ext, int B_) : B(B_) {
        read_range(ext, ymin, ymax);
        range = __dsub_rn(ymax, ymin);
        ymin32 = (float)ymin;
        sc32 = range > 0.0 ? (float)((double)B / range) : 0.f;
    }
    __device__ __forceinline__ int32_t operator()(double yv) const {
        if (!(range > 0.0)) return 0;
        const float y32 = (float)yv;
        const float t32 = (y32 - ymin32) * sc32;
        const float fl32 = floorf(t32);
        const float eps = 0x1p-21f * ((fabsf(y32) + fabsf(ymin32)) * sc32 * 2.f + fabsf(t32)) + 0x1p-60f;
        int32_t b;
        if (t32 - fl32 > eps && fl32 + 1.f - t32 > eps) {
            b = (int32_t)fl32;
        } else {
            const double t = __ddiv_rn(__dsub_rn(yv, ymin), range);
            b = (int32_t)floor(__dmul_rn(t, (double)B));
        }
        b = b > B - 1 ? B - 1 : b;
        return b < 0 ? 0 : b;
    }
};

// Bins of a 1-D grid, counted per (bin, warp tile) for the stable counting
// sort that gives the model matrix's CSR form.  The CTA has blockDim.x / 32
// warps, each owning one tile of kSortTile points.
__global__ void k_bins_count(const double *__restrict__ y, int64_t N, int B,
                             const unsigned long long *ext, int32_t *__restrict__ bins,
                             int32_t *__restrict__ counts, int64_t n_tiles) {
    extern __shared__ int32_t s_cnt[];  // [warps][B]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *cnt = s_cnt + warp * B;
    for (int b = lane; b < B; b += 32) cnt[b] = 0;
    __syncwarp();
    const int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const BinRule rule(ext, B);
    if (tile < n_tiles) {
        const int64_t i0 = tile * kSortTile;
        const int64_t i1 = min(N, i0 + kSortTile);
        for (int64_t i = i0 + lane; i < i1; i += 32) {
            const int32_t b = rule(y[i]);
            bins[i] = b;
            atomicAdd(&cnt[b], 1);
        }
        __syncwarp();
        for (int b = lane; b < B; b += 32) counts[(int64_t)b * n_tiles + tile] = cnt[b];
    }
}

// Bins of a 2-D / 3-D grid (its histogram layouts sort their own keys):
// grid-stride over pairs of points, and the power tables' reference point
// and scales from the first thread.
__global__ void k_bins_scale(const double *__restrict__ y, int64_t N, int B, const unsigned long long *ext,
                             int32_t *__restrict__ bins, double *s_out) {
    pdl_trigger();
    pdl_wait();
    const BinRule rule(ext, B);
    if (blockIdx.x == 0 && threadIdx.x == 0) write_scale(rule.ymin, rule.ymax, N, s_out);
    const int64_t n2 = N >> 1;
    const double2 *y2 = reinterpret_cast<const double2 *>(y);
    int2 *b2 = reinterpret_cast<int2 *>(bins);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = y2[i];
        b2[i] = make_int2(rule(v.x), rule(v.y));
    }
    if ((N & 1) && blockIdx.x == 0 && threadIdx.x == 0) bins[N - 1] = rule(y[N - 1]);
}

// Grid-wide barrier of a cooperative launch (every block resident): one
// counter, zeroed before the launch, that every block increments once; the
// wait is bounded (the device status records an expired wait and the
// caller's blocks return false).
constexpr uint32_t kGridSpin = 1u << 22;
__device__ __forceinline__ bool grid_barrier(unsigned long long *ctr, int *dstatus) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1ull);
        int ok = 1;
        for (uint32_t i = 0; *reinterpret_cast<volatile unsigned long long *>(ctr) < gridDim.x; ++i) {
            if (i > kGridSpin) {
                atomicCAS(dstatus, 0, VUP_DSTAT_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Model evaluation and bins of a separable built-in model on a 2-D / 3-D
// grid in one cooperative launch: y and its exact range (as k_model_combine),
// a grid-wide barrier, then the bins (Eq. 4, as k_bins_scale) from the
// values each thread kept, and the power-table scale.  ext[2] is the barrier
// counter.  With zh / zl given, also the contraction's split BF16 power table
// of the rest-row orientation (as k_power_table_bf16<true>: y[rest * R + red]
// -> [rest * 4 + j][red], row stride ld, zeros in the padding up to Qext rests
// and ld reds).
constexpr int kKeepY = 8;  // values of y a thread keeps in registers across the barrier
__global__ void __launch_bounds__(256) k_model_bins(double *__restrict__ y, int64_t N, GridGeom G, int model,
                                                    Theta th, const double2 *__restrict__ terms,
                                                    unsigned long long *ext, int B, int32_t *__restrict__ bins,
                                                    double *s_out, int *dstatus, __nv_bfloat16 *__restrict__ zh,
                                                    __nv_bfloat16 *__restrict__ zl, int64_t R, int64_t ld,
                                                    int64_t Qext) {
    pdl_trigger();
    pdl_wait();
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, step = (int64_t)gridDim.x * blockDim.x;
    double keep[kKeepY];
    unsigned long long mn = ~0ull, mx = 0ull;
    IndexWalk w(G, i0, step);
    auto value = [&](int64_t i) {
        const double v = combine_terms(w.a, G, model, th, terms);
        w.next();
        y[i] = v;
        const unsigned long long kv = dkey(v);
        mn = kv < mn ? kv : mn;
        mx = kv > mx ? kv : mx;
        return v;
    };
#pragma unroll
    for (int q = 0; q < kKeepY; ++q) {
        const int64_t i = i0 + q * step;
        keep[q] = i < N ? value(i) : 0.0;
    }
    for (int64_t i = i0 + kKeepY * step; i < N; i += step) value(i);
    range_reduce(mn, mx, ext);
    if (!grid_barrier(ext + 2, dstatus)) return;
    const BinRule rule(ext, B);
    if (blockIdx.x == 0 && threadIdx.x == 0) write_scale(rule.ymin, rule.ymax, N, s_out);
    double zc, zs, zsa;
    power_ref(rule.ymin, rule.ymax, zc, zs, zsa);
    const double inv = 1.0 / zs;  // z = (y - c) / s
    const float pf = (float)power_factor(N);  // tables hold z^j 2^e
    IndexWalk w2(G, i0, step);  // red = the last axis, rest = the other axes' flat index
    auto table = [&](double v) {
        const int64_t rest = G.ndim == 3 ? (int64_t)w2.a[0] * G.n[1] + w2.a[1] : w2.a[0];
        const int64_t red = G.ndim == 3 ? w2.a[2] : w2.a[1];
        w2.next();
        const float z = (float)__dmul_rn(__dsub_rn(v, zc), inv);
        float p = z * pf;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j) p *= z;
            const __nv_bfloat16 hh = __float2bfloat16_rn(p);
            const int64_t idx = (rest * 4 + j) * ld + red;
            zh[idx] = hh;
            zl[idx] = __float2bfloat16_rn(p - __bfloat162float(hh));
        }
    };
#pragma unroll
    for (int q = 0; q < kKeepY; ++q) {
        const int64_t i = i0 + q * step;
        if (i < N) {
            bins[i] = rule(keep[q]);
            if (zh) table(keep[q]);
        }
    }
    for (int64_t i = i0 + kKeepY * step; i < N; i += step) {
        const double v = y[i];
        bins[i] = rule(v);
        if (zh) table(v);
    }
    if (zh) {
        // padding: reds R .. ld of every rest, and every red of rests Q .. Qext
        const int64_t Q = N / R, pad_r = ld - R, n_pad = Q * pad_r + (Qext - Q) * ld;
        for (int64_t e = i0; e < n_pad * 4; e += step) {
            const int64_t c = e >> 2, j = e & 3;
            int64_t rest, red;
            if (c < Q * pad_r) {
                rest = c / pad_r;
                red = R + (c - rest * pad_r);
            } else {
                const int64_t c2 = c - Q * pad_r;
                rest = Q + c2 / ld;
                red = c2 - (rest - Q) * ld;
            }
            const int64_t idx = (rest * 4 + j) * ld + red;
            zh[idx] = __float2bfloat16_rn(0.f);
            zl[idx] = __float2bfloat16_rn(0.f);
        }
    }
}

// A kernel of the key-sorted streams' build returns at once when the device
// found the record stream cheaper than either of them (gate 0).
__device__ __forceinline__ bool gated_off(const int32_t *gate) { return gate && gate[0] == 0; }

// Points per (key, warp tile) of a key array with key < Bk.
__global__ void k_count(const int32_t *__restrict__ keys, int64_t N, int Bk, int32_t *__restrict__ counts,
                        int64_t n_tiles, const int32_t *gate) {
    if (gated_off(gate)) return;
    extern __shared__ int32_t s_cnt[];  // [warps][Bk]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *cnt = s_cnt + warp * Bk;
    for (int b = lane; b < Bk; b += 32) cnt[b] = 0;
    __syncwarp();
    const int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (tile < n_tiles) {
        const int64_t i0 = tile * kSortTile;
        const int64_t i1 = min(N, i0 + kSortTile);
        for (int64_t i = i0 + lane; i < i1; i += 32) atomicAdd(&cnt[keys[i]], 1);
        __syncwarp();
        for (int b = lane; b < Bk; b += 32) counts[(int64_t)b * n_tiles + tile] = cnt[b];
    }
}

// ---- histogram layout ---------------------------------------------------------
// A layout gathers one axis per point from a shared-memory factor tile (the
// last axis, or on 2-D grids axis 0) and cuts it into P parts of part_rows
// rows; its flat order puts the gathered index innermost.  Both candidate
// geometries travel to the kernels and the device-side choice sel[0] picks
// one, so only the chosen layout is sorted and walked.
struct LayGeom {
    int64_t n_last, part_rows;
    int P;
};
struct LaySel {
    LayGeom g[2];
    const int32_t *sel;
    __device__ __forceinline__ LayGeom get() const { return g[sel[0] ? 1 : 0]; }
};

// Intervals of both 2-D layouts (stretches of one (part, bin) key along the
// gathered axis), counted without sorting: 1 + key changes along each line.
__global__ void k_iv_count(const int32_t *__restrict__ bins, int64_t n0, int64_t n1, int B, LaySel L,
                           int32_t *__restrict__ cnt) {
    const int64_t N = n0 * n1;
    int32_t c0 = 0, c1 = 0;
    const uint32_t p0 = (uint32_t)L.g[0].part_rows, p1 = (uint32_t)L.g[1].part_rows;
    const uint32_t m1 = (uint32_t)n1;  // N < 2^31: 32-bit index arithmetic
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i0 = (uint32_t)i / m1, i1 = (uint32_t)i - i0 * m1;
        const int32_t b = bins[i];
        // layout 0 gathers axis 1, layout 1 axis 0
        c0 += i1 == 0 || (i1 / p0) * B + b != ((i1 - 1) / p0) * B + bins[i - 1];
        c1 += i0 == 0 || (i0 / p1) * B + b != ((i0 - 1) / p1) * B + bins[i - n1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_xor_sync(0xffffffffu, c0, o);
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&cnt[0], c0);
        atomicAdd(&cnt[1], c1);
    }
}

// Layout choice: the one with fewer intervals (both streams' work grows with
// the runs and intervals of the layout, and a layout's runs are at most its
// intervals).
__global__ void k_pick_layout(const int32_t *cnt, int32_t *sel) { sel[0] = cnt[1] < cnt[0] ? 1 : 0; }

// Sort keys of the chosen layout: key = part of the gathered index * B + bin,
// in the layout's flat order.  bins is viewed as an [R][C] matrix (C = the
// last axis); layout 1 (2-D) walks its transpose.  32 x 32 tiles go through
// shared memory so that reads and writes are coalesced either way.
__global__ void k_layout_keys(const int32_t *__restrict__ bins, int64_t R, int64_t C, int B, LaySel L,
                              int32_t *__restrict__ keys, const int32_t *gate) {
    if (gated_off(gate)) return;
    __shared__ int32_t t[32][33];
    const bool tr = L.sel[0] != 0;  // uniform over the grid
    const LayGeom G = L.get();
    const int64_t cb = (int64_t)blockIdx.x * 32;
    for (int64_t rb = (int64_t)blockIdx.y * 32; rb < R; rb += (int64_t)gridDim.y * 32) {
        for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
            const int64_t r = rb + yy, c = cb + threadIdx.x;
            if (r < R && c < C) {
                const int32_t b = bins[r * C + c];
                if (tr) t[yy][threadIdx.x] = (int32_t)(r / G.part_rows) * B + b;
                else keys[r * C + c] = (int32_t)(c / G.part_rows) * B + b;
            }
        }
        if (!tr) continue;
        __syncthreads();
        for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
            const int64_t c = cb + yy, r = rb + threadIdx.x;
            if (r < R && c < C) keys[c * R + r] = t[threadIdx.x][yy];
        }
        __syncthreads();
    }
}

// Whether the key-sorted point and interval streams are built (sel[4]): not
// when the record stream costs less than the interval stream and less than
// any point stream can (4 per point, the runs' share not counted), unless a
// caller asked for one of them.  The record stream is then chosen at once
// (sel[1] = 2, before the rest of the layout is built); otherwise the choice
// waits for the run counts (sel[1] = -1 meanwhile) and is one of the others.
__global__ void k_need_keys(const int32_t *n_rec, const int32_t *n_iv, int64_t N, int nf, int force,
                            int force_keys, int32_t *sel, int32_t *n_runs) {
    const int64_t c_iv = 19 * (int64_t)n_iv[0];
    const int64_t c_rec = (16 + 6 * nf) * (int64_t)n_rec[0] + 6 * ((int64_t)n_iv[0] + 2 * (int64_t)n_rec[0]);
    const int need = force_keys || force == 0 || force == 1 || (force < 0 && !(c_rec < 4 * N && c_rec <= c_iv));
    sel[4] = need;
    sel[1] = need ? -1 : 2;
    if (!need) n_runs[0] = 0;  // no point stream built
}

// Stream costs, in units of about 3.3 ps of kernel time per 128-density tile
// (fitted to measured launches on 2-D and 3-D grids): point stream 4 per
// point (one gather) + 20 per run (rest-factor pipeline); interval stream 19
// per interval (two gathers, a difference, a rest-factor load); record stream
// 16 + 6 per extra rest axis per record (record words, one rest-factor load
// per rest axis, the group flushes) + 6 per prefix-sum gather (a record gathers
// 1 + 4 per half-group holding a bin: about m + 2 for m bins, m summing to the
// interval count).  After the key sort: the point or the
// interval stream, whichever costs less (unless forced), when the record
// stream was not chosen before it.
__global__ void k_pick_stream(const int32_t *n_runs, const int32_t *n_iv, int64_t N, int force, int32_t *sel) {
    if (sel[4] == 0) return;  // the record stream, chosen before the key sort
    const int64_t c_pt = 4 * N + 20 * (int64_t)n_runs[0];
    const int64_t c_iv = 19 * (int64_t)n_iv[0];
    sel[1] = (force == 0 || force == 1) ? force : (c_iv < c_pt ? 1 : 0);
}

// Stable scatter: each warp walks its tile in order, 32 points at a time;
// equal keys inside a step are ranked by lane with __match_any_sync.
__global__ void k_sort_scatter(const int32_t *__restrict__ keys, int64_t N, int Bk, const int32_t *gate,
                               const int32_t *__restrict__ starts, int64_t n_tiles,
                               int32_t *__restrict__ perm) {
    if (gated_off(gate)) return;
    extern __shared__ int32_t s_cnt[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *cnt = s_cnt + warp * Bk;
    const int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (tile >= n_tiles) return;
    for (int b = lane; b < Bk; b += 32) cnt[b] = starts[(int64_t)b * n_tiles + tile];
    __syncwarp();
    const int64_t i0 = tile * kSortTile;
    const int64_t i1 = min(N, i0 + kSortTile);
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t base = i0; base < i1; base += 32) {
        const int64_t i = base + lane;
        const bool v = i < i1;
        const unsigned act = __ballot_sync(0xffffffffu, v);
        int32_t b = v ? keys[i] : -1;
        unsigned peers = __match_any_sync(0xffffffffu, b);
        peers &= act;
        int32_t pos = 0;
        if (v) {
            pos = cnt[b] + __popc(peers & lt);
            perm[pos] = (int32_t)i;
        }
        __syncwarp();
        if (v && (peers & lt) == 0) cnt[b] += __popc(peers);
        __syncwarp();
    }
}

// ---- exclusive scan (three-phase, deterministic), int32 or int64 -----------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *s_warp, T &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : T(0);
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    T warp_off = warp > 0 ? s_warp[warp - 1] : T(0);
    total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + x - v;
}

template <typename T>
__global__ void k_scan_blocks(const T *__restrict__ in, T *__restrict__ out, int64_t L, T *__restrict__ block_sums,
                              const int32_t *gate) {
    if (gated_off(gate)) return;
    __shared__ T s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T tsum = 0;
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < L ? in[base + j] : T(0);
        tsum += v[j];
    }
    T total;
    T off = block_excl_scan(tsum, s_warp, total);
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < L) out[base + j] = off;
        off += v[j];
    }
    if (threadIdx.x == 0 && block_sums) block_sums[blockIdx.x] = total;
}

template <typename T>
__global__ void k_scan_add(T *__restrict__ out, int64_t L, const T *__restrict__ block_off, const int32_t *gate) {
    if (gated_off(gate)) return;
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    const T add = block_off[blockIdx.x];
    for (int j = threadIdx.x; j < kScanBlock; j += blockDim.x)
        if (base + j < L) out[base + j] += add;
}

// ---- runs, intervals and chunks of the segmented histogram ------------------
// A run is a maximal stretch of sorted points sharing the sort key (part and
// bin) and every axis index but the gathered one; an interval is a maximal
// stretch of a run whose gathered rows are consecutive (the points of one bin
// along one line of the grid).  One flag word per sorted point holds both
// start flags (run: bit 0, interval: bit 32), so a single 64-bit scan numbers
// runs (low half) and intervals (high half).
__global__ void k_layout_flags(const int32_t *__restrict__ perm, const int32_t *__restrict__ keys, int64_t N,
                               LaySel L, unsigned long long *__restrict__ flags, const int32_t *gate) {
    if (gated_off(gate)) return;
    const int64_t n_last = L.get().n_last;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
         t += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long f = 1ull | (1ull << 32);
        if (t > 0) {
            const int32_t i = perm[t], ip = perm[t - 1];
            const bool run = keys[i] != keys[ip] || i / n_last != ip / n_last;
            const bool iv = run || i != ip + 1;  // same line: consecutive gathered rows
            f = (run ? 1ull : 0ull) | (iv ? 1ull << 32 : 0ull);
        }
        flags[t] = f;
    }
}

// Per sorted point t: the run arrays at run starts; hpt[t] = the point's row
// inside its part (<< shift: its byte offset in a shared-memory tile of
// 2^shift-byte rows, kRowBits wide -- rows past that field only occur with
// parts too large for a tile, whose kernel reads the row from the sorted
// order instead) | run-end / key-end flags (bits 30, 31); the interval words
// (first row << shift; (last row + 1) << shift | the flags of its last point)
// and each interval's rest index.
__global__ void k_layout_build(const int32_t *__restrict__ perm, const int32_t *__restrict__ keys, int64_t N,
                               LaySel L, int shift, const unsigned long long *__restrict__ flags,
                               const unsigned long long *__restrict__ excl, int32_t *__restrict__ run_start,
                               int32_t *__restrict__ run_rest, int32_t *__restrict__ run_bin,
                               uint32_t *__restrict__ hpt, int32_t *__restrict__ n_runs, uint2 *__restrict__ ipt,
                               int32_t *__restrict__ iv_rest, int32_t *__restrict__ n_iv, const int32_t *gate) {
    if (gated_off(gate)) return;
    const LayGeom G = L.get();
    const uint32_t rmask = (1u << kRowBits) - 1u;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = perm[t];
        const unsigned long long f = flags[t], e = excl[t];
        const int32_t run_f = (int32_t)(f & 1ull), iv_f = (int32_t)(f >> 32);
        const int32_t rid = (int32_t)(e & 0xffffffffull) + run_f - 1;
        const int32_t iid = (int32_t)(e >> 32) + iv_f - 1;
        const int32_t key = keys[i];
        const int32_t rest = (int32_t)(i / G.n_last);
        if (run_f) {
            run_start[rid] = (int32_t)t;
            run_rest[rid] = rest;
            run_bin[rid] = key;
        }
        const bool end = t == N - 1;
        const unsigned long long fn = end ? (1ull | (1ull << 32)) : flags[t + 1];
        const bool last = (fn & 1ull) != 0, iv_last = (fn >> 32) != 0;
        const bool key_last = end || keys[perm[t + 1]] != key;
        const int64_t a = i - (int64_t)rest * G.n_last;
        const uint32_t row = (uint32_t)(a - (a / G.part_rows) * G.part_rows) & rmask;
        const uint32_t fl = (last ? kRunEnd : 0u) | (key_last ? kBinEnd : 0u);
        hpt[t] = (row << shift) | fl;
        uint32_t *w = reinterpret_cast<uint32_t *>(ipt + iid);
        if (iv_f) {
            w[0] = row << shift;
            iv_rest[iid] = rest;
        }
        if (iv_last) w[1] = (((row + 1u) & rmask) << shift) | fl;
        if (end) {
            n_runs[0] = rid + 1;
            run_start[rid + 1] = (int32_t)N;
            n_iv[0] = iid + 1;
        }
    }
}

// The run-end word of run r (and the word pair of interval i) also carries
// the rest-axis index of run r + 4 (interval i + 4): the histogram kernel
// loads that factor four ahead.  The code sits in the 21 bits beside the row
// field: `shift` low bits (0 .. shift-1) and 30 - shift - kRowBits high bits
// (shift + kRowBits .. 29).  2-D grids split the rest index itself; 3-D grids
// put a0 in the low field and a1 in the high field.  Zero past the end.
constexpr int kRunAhead = 4;
__device__ __forceinline__ uint32_t rest_code(int32_t rest, int ndim, int64_t n1, int shift) {
    const uint32_t lo_mask = (1u << shift) - 1u;
    const uint32_t hi_mask = (1u << (30 - shift - kRowBits)) - 1u;
    uint32_t lo, hi;
    if (ndim == 3) {
        lo = (uint32_t)(rest / n1);
        hi = (uint32_t)(rest % n1);
    } else {
        lo = (uint32_t)rest & lo_mask;
        hi = (uint32_t)rest >> shift;
    }
    return (lo & lo_mask) | ((hi & hi_mask) << (shift + kRowBits));
}
__global__ void k_layout_encode(const int32_t *__restrict__ run_start, const int32_t *__restrict__ run_rest,
                                const int32_t *__restrict__ n_runs_p, const int32_t *__restrict__ iv_rest,
                                const int32_t *__restrict__ n_iv_p, int ndim, int64_t n1, int shift,
                                uint32_t *__restrict__ hpt, uint2 *__restrict__ ipt, int run_ahead,
                                const int32_t *gate) {
    if (gated_off(gate)) return;
    const int32_t n_runs = n_runs_p[0], n_iv = n_iv_p[0];
    const int32_t n = n_runs > n_iv ? n_runs : n_iv;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t xr = x + run_ahead, xa = x + kRunAhead;
        if (x < n_runs && xr < n_runs) hpt[run_start[x + 1] - 1] |= rest_code(run_rest[xr], ndim, n1, shift);
        if (x < n_iv && xa < n_iv) reinterpret_cast<uint32_t *>(ipt + x)[1] |= rest_code(iv_rest[xa], ndim, n1, shift);
    }
}

// Chunks, C per part: chunk c of part p starts at the first run whose first
// point is >= lo_p + (hi_p - lo_p) c / C, [lo_p, hi_p) being the part's
// points; chunk_iv[c] is its first interval (chunks start on runs, which
// start intervals).  Entry P C is the end.
__global__ void k_chunks(const int32_t *__restrict__ run_start, const int32_t *__restrict__ n_runs_p,
                         const int32_t *__restrict__ koff, int B, LaySel L, int C,
                         const unsigned long long *__restrict__ excl, int64_t N, const int32_t *__restrict__ n_iv_p,
                         int32_t *__restrict__ chunk_pt, int32_t *__restrict__ chunk_run,
                         int32_t *__restrict__ chunk_iv, const int32_t *gate) {
    if (gated_off(gate)) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = L.get().P;
    if (c > P * C) return;
    const int32_t n_runs = n_runs_p[0];
    int32_t r;
    if (c == P * C) {
        r = n_runs;
    } else {
        const int p = c / C, cc = c - p * C;
        const int64_t lo = koff[p * B], hi = koff[(p + 1) * B];
        const int64_t target = lo + ((hi - lo) * (int64_t)cc) / C;
        int32_t a = 0, b = n_runs;  // first r in [0, n_runs] with run_start[r] >= target
        while (a < b) {
            int32_t mid = (a + b) >> 1;
            if (run_start[mid] >= target) b = mid; else a = mid + 1;
        }
        r = a;
    }
    const int32_t pt = run_start[r];
    chunk_run[c] = r;
    chunk_pt[c] = pt;
    chunk_iv[c] = pt < N ? (int32_t)(excl[pt] >> 32) : n_iv_p[0];
}

// Key offsets of a counting sort: koff[b] = starts[b * n_tiles], koff[Bk] = N.
__global__ void k_koff(const int32_t *__restrict__ starts, int64_t n_tiles, int Bk, int64_t N,
                       int32_t *__restrict__ koff, const int32_t *gate) {
    if (gated_off(gate)) return;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < Bk) koff[b] = starts[(int64_t)b * n_tiles];
    else if (b == Bk) koff[b] = (int32_t)N;
}

__global__ void k_chunk_bins(const int32_t *__restrict__ chunk_run, const int32_t *__restrict__ run_bin, LaySel L,
                             int C, int32_t *__restrict__ chunk_bin, const int32_t *gate) {
    if (gated_off(gate)) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.get().P * C) return;
    const int32_t r0 = chunk_run[c], r1 = chunk_run[c + 1];
    chunk_bin[2 * c] = r1 > r0 ? run_bin[r0] : -1;
    chunk_bin[2 * c + 1] = r1 > r0 ? run_bin[r1 - 1] : -1;
}

// First and last chunk holding points of each key (-1, -1 for an empty key):
// chunk c holds the points [chunk_pt[c], chunk_pt[c + 1]).
__device__ __forceinline__ int chunk_holding(const int32_t *chunk_pt, int n, int32_t pt) {
    int lo = 0, hi = n;  // last c in [0, n) with chunk_pt[c] <= pt
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (chunk_pt[mid] <= pt) lo = mid; else hi = mid;
    }
    return lo;
}
__global__ void k_key_chunks(const int32_t *__restrict__ koff, LaySel L, int B, const int32_t *__restrict__ chunk_pt,
                             int C, int2 *__restrict__ out, const int32_t *gate) {
    if (gated_off(gate)) return;
    const int key = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = L.get().P;
    if (key >= P * B) return;
    const int n_chunks = P * C;
    const int32_t o0 = koff[key], o1 = koff[key + 1];
    out[key] = o0 == o1 ? make_int2(-1, -1)
                        : make_int2(chunk_holding(chunk_pt, n_chunks, o0), chunk_holding(chunk_pt, n_chunks, o1 - 1));
}

// ---- record stream ------------------------------------------------------------
// A record is a stretch of one line (every axis but the gathered one fixed)
// inside one part whose points fall in one group of kRecBins consecutive bins
// and whose bins change monotonically along the gathered axis.  Each bin of
// the group then holds one sub-range of the stretch, and nine boundaries
// B_0..B_8 describe them all: bin 8q + j holds rows [B_j, B_j+1) when the
// bins rise along the line, [B_j+1, B_j) when they fall (the record's sign),
// an empty range (B_j+1 = B_j) when absent.  The histogram adds sign f_rest
// (P[B_j+1] - P[B_j]) to each bin present: m + 1 prefix-sum gathers and one
// rest-factor load for a record over m bins, where the interval stream needs
// two gathers and a load per bin.  Records come from the intervals in line
// order (maximal stretches of one key along a line): a record starts at a
// line-part start, a group change, or where the bin steps change sign inside
// a group.
constexpr int kRecBins = 8;
constexpr uint32_t kRecNeg = 1u << 30;  // bins fall along the line

constexpr uint32_t kRecEnd = 1u << 31;  // last record of its group

// The record stream, one thread per (part, line) segment of the chosen layout
// (records never cross one), walking the bins in place in row order: an
// interval starts at the segment's first row or where the bin changes; a
// record starts at an interval whose group differs from the interval before
// it, or whose bin step turns against the step before it when the three
// intervals share a group.  Each record goes to the segment's slots
// tmp[seg * cap + i] with its group and its rank among the segment's records
// of that group; cnt[group * NL + line] counts the records of every (group,
// line) and n_iv the intervals.  bins is viewed as [R][C], C the last axis;
// layout 1 (2-D) walks the columns.  A record's boundary rows B_0..B_8 (rows
// inside the part): bin 8q + j holds rows [B_j, B_j+1) when the bins rise
// along the line, [B_j+1, B_j) when they fall.
struct RecGeom {
    int64_t R, C;
    int GB;       // groups of kRecBins bins per part
    int64_t NL;   // line stride of the count matrix (the most lines of either layout)
    int64_t cap;  // slots per segment (the most part rows)
    int ndim;
    int64_t n1;   // 3-D rest code: line = a0 n1 + a1 -> a0 | a1 << 15
};

constexpr int kWalkWarps = 8;  // segments (warps) per block of the record walk
__global__ void __launch_bounds__(kWalkWarps * 32) k_rec_walk(const int32_t *__restrict__ bins, RecGeom Q, LaySel L,
                                                              int32_t *__restrict__ cnt, int32_t *__restrict__ n_iv,
                                                              uint4 *__restrict__ tmp, int32_t *__restrict__ seg_n) {
    extern __shared__ int32_t s_rank[];  // [warps][GB]: records so far of each group of the part
    const bool tr = L.sel[0] != 0;
    const LayGeom G = L.get();
    const int64_t n_lines = tr ? Q.C : Q.R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // one warp per segment; the warps of a block walk consecutive lines of one part
    const int64_t seg = (int64_t)blockIdx.x * kWalkWarps + warp;
    if (seg >= (int64_t)G.P * n_lines) return;
    const int p = (int)(seg / n_lines);
    const int64_t line = seg - (int64_t)p * n_lines;
    const int64_t row0 = (int64_t)p * G.part_rows, row1 = min(G.n_last, row0 + G.part_rows);
    int32_t *rank = s_rank + warp * Q.GB;
    for (int q = lane; q < Q.GB; q += 32) rank[q] = 0;
    __syncwarp();
    const int64_t stride = tr ? Q.C : 1;
    const int32_t *src = bins + (tr ? line : line * Q.C);
    uint4 *slot = tmp + 2 * seg * Q.cap;

    // record state, the same in every lane; lane j < 8 holds st_j, the first
    // row (relative to row0) of bin 8 rq + j in the open record, -1 if absent
    int32_t b1 = -1, b2 = -1;  // bins of the current interval and of the one before it
    int rq = -1, dir = 0, rprev = -1;
    int32_t st = -1;
    int32_t niv = 0, nrec = 0;
    auto emit = [&](int64_t e_row) {
        const int32_t e = (int32_t)(e_row - row0);
        // B_j: the least first row among the bins at or above j (rising) or
        // below j (falling), e if none -- a suffix / prefix minimum over lanes
        const int32_t mine = (lane < kRecBins && st >= 0) ? st : e;
        int32_t w = mine;
        if (dir >= 0) {
#pragma unroll
            for (int o = 1; o < kRecBins; o <<= 1) {
                const int32_t t = __shfl_down_sync(0xffffffffu, w, o);
                if (lane + o < kRecBins) w = min(w, t);
            }
        } else {
            int32_t x = __shfl_up_sync(0xffffffffu, mine, 1);  // exclusive: bins below j
            x = lane == 0 ? e : x;
            w = x;
#pragma unroll
            for (int o = 1; o < kRecBins + 1; o <<= 1) {
                const int32_t t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w = min(w, t);
            }
        }
        if (lane > kRecBins) w = 0;
        // lanes 0, 2, 4, 6 pack (B_j, B_j+1); lane 8 holds B_8
        const uint32_t pair = (uint32_t)w | ((uint32_t)__shfl_down_sync(0xffffffffu, w, 1) << 16);
        const uint32_t u0 = __shfl_sync(0xffffffffu, pair, 0), u1 = __shfl_sync(0xffffffffu, pair, 2),
                       u2 = __shfl_sync(0xffffffffu, pair, 4), u3 = __shfl_sync(0xffffffffu, pair, 6);
        const uint32_t w8 = (uint32_t)__shfl_sync(0xffffffffu, w, kRecBins);
        if (lane == 0) {
            const int32_t g = p * Q.GB + rq;
            const int32_t r = rank[rq]++;
            slot[2 * nrec] = make_uint4(u0, u1, u2, u3);
            slot[2 * nrec + 1] = make_uint4(w8 | (dir < 0 ? kRecNeg : 0u), (uint32_t)line, (uint32_t)g, (uint32_t)r);
        }
        __syncwarp();
        ++nrec;
    };
    int32_t carry = -1;  // bin of the row before the window
    for (int64_t r0w = row0; r0w < row1; r0w += 32) {
        const int64_t r = r0w + lane;
        const int32_t b = r < row1 ? src[r * stride] : -1;
        int32_t bp = __shfl_up_sync(0xffffffffu, b, 1);
        if (lane == 0) bp = carry;
        uint32_t starts = __ballot_sync(0xffffffffu, r < row1 && b != bp);
        carry = __shfl_sync(0xffffffffu, b, 31);
        while (starts) {
            const int L = __ffs(starts) - 1;
            starts &= starts - 1;
            const int32_t bi = __shfl_sync(0xffffffffu, b, L);
            const int64_t ri = r0w + L;
            ++niv;
            const int q = bi / kRecBins;
            bool start;
            if (b1 < 0 || q != b1 / kRecBins) start = true;
            else if (b2 >= 0 && b2 / kRecBins == q) start = ((bi - b1) > 0) != ((b1 - b2) > 0);
            else start = false;
            if (start) {
                if (rq >= 0) emit(ri);
                rq = q;
                dir = 0;
                rprev = -1;
                st = -1;
            }
            if (lane == bi - q * kRecBins) st = (int32_t)(ri - row0);
            if (rprev >= 0 && dir == 0) dir = bi > rprev ? 1 : -1;
            rprev = bi;
            b2 = b1;
            b1 = bi;
        }
    }
    if (rq >= 0) emit(row1);
    __syncwarp();
    for (int q = lane; q < Q.GB; q += 32)
        if (rank[q]) cnt[((int64_t)p * Q.GB + q) * Q.NL + line] = rank[q];
    if (lane == 0) {
        seg_n[seg] = nrec;
        atomicAdd(n_iv, niv);
    }
}

// Every record from its segment slot to its place in (group, line, row)
// order (starts: the exclusive scan of the (group, line) counts): words (B_0 |
// B_1 << 16, .., B_6 | B_7 << 16) and (B_8 | sign | group end, rest code of
// the record kRunAhead places later, group, 0), and its rest index (the
// line).  One warp per segment.
__global__ void k_rec_scatter(const uint4 *__restrict__ tmp, const int32_t *__restrict__ seg_n, RecGeom Q,
                              LaySel L, const int32_t *__restrict__ starts, const int32_t *__restrict__ goff,
                              const int32_t *__restrict__ n_rec_p, uint4 *__restrict__ rec,
                              int32_t *__restrict__ rec_rest) {
    const bool tr = L.sel[0] != 0;
    const LayGeom G = L.get();
    const int64_t n_seg = (int64_t)G.P * (tr ? Q.C : Q.R);
    const int32_t n_rec = n_rec_p[0];
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (w0 == 0 && lane < 16) {  // the records past the last read as empty
        rec[2 * ((int64_t)n_rec + lane)] = make_uint4(0u, 0u, 0u, 0u);
        rec[2 * ((int64_t)n_rec + lane) + 1] = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int64_t sg = w0; sg < n_seg; sg += nw) {
        const int32_t n = seg_n[sg];
        const uint4 *slot = tmp + 2 * sg * Q.cap;
        for (int32_t i = lane; i < n; i += 32) {
            const uint4 u = slot[2 * i], v = slot[2 * i + 1];
            const uint32_t line = v.y, g = v.z;
            const int64_t pos = (int64_t)starts[(int64_t)g * Q.NL + line] + v.w;
            rec[2 * pos] = u;
            uint32_t *w1 = reinterpret_cast<uint32_t *>(rec + 2 * pos + 1);
            w1[0] = v.x | (pos + 1 == goff[g + 1] ? kRecEnd : 0u);
            if (pos + kRunAhead >= n_rec) w1[1] = 0u;
            w1[2] = g;
            w1[3] = 0u;
            const uint32_t code =
                Q.ndim == 3 ? (uint32_t)(line / Q.n1) | ((uint32_t)(line % Q.n1) << 15) : (uint32_t)line;
            if (pos >= kRunAhead) reinterpret_cast<uint32_t *>(rec + 2 * (pos - kRunAhead) + 1)[1] = code;
            rec_rest[pos] = (int32_t)line;
        }
    }
}

// First record of every group (n_groups + 2 entries: the last two = the
// record count) from the scanned (group, line) counts.
__global__ void k_rec_goff(const int32_t *__restrict__ starts, const int32_t *__restrict__ counts, int64_t Lr,
                           int64_t NL, int n_groups, int32_t *__restrict__ goff, int32_t *__restrict__ n_rec) {
    const int32_t total = starts[Lr - 1] + counts[Lr - 1];
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n_groups + 2; g += gridDim.x * blockDim.x)
        goff[g] = g < n_groups ? starts[g * NL] : total;
    if (blockIdx.x == 0 && threadIdx.x == 0) n_rec[0] = total;
}

// Record chunks, C per part (equal record counts; records cost alike):
// chunk c of part p starts at record lo_p + (hi_p - lo_p) c / C; its first and
// last groups (-1 when empty); entry P C is the end.  A group may be cut by
// chunk bounds, like a key of the point stream.
__global__ void k_rec_chunks(const int32_t *__restrict__ goff, const int32_t *__restrict__ n_rec_p, int GB,
                             LaySel L, int C, const uint4 *__restrict__ rec, int32_t *__restrict__ chunk_rec,
                             int32_t *__restrict__ chunk_grp) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = L.get().P;
    if (c > P * C) return;
    int32_t r;
    if (c == P * C) {
        r = n_rec_p[0];
    } else {
        const int p = c / C, cc = c - p * C;
        const int64_t lo = goff[p * GB], hi = goff[(p + 1) * GB];
        r = (int32_t)(lo + ((hi - lo) * (int64_t)cc) / C);
    }
    chunk_rec[c] = r;
    if (c < P * C) {
        const int p = c / C, cc = c - p * C;
        const int64_t lo = goff[p * GB], hi = goff[(p + 1) * GB];
        const int32_t r1 = (int32_t)(lo + ((hi - lo) * (int64_t)(cc + 1)) / C);
        chunk_grp[2 * c] = r1 > r ? (int32_t)rec[2 * (int64_t)r + 1].z : -1;
        chunk_grp[2 * c + 1] = r1 > r ? (int32_t)rec[2 * (int64_t)(r1 - 1) + 1].z : -1;
    }
}

// First and last chunk holding records of each group (-1, -1 for an empty group).
__global__ void k_rec_group_chunks(const int32_t *__restrict__ goff, int n_groups,
                                   const int32_t *__restrict__ chunk_rec, LaySel L, int C, int2 *__restrict__ out) {
    const int gr = blockIdx.x * blockDim.x + threadIdx.x;
    if (gr >= n_groups) return;
    const int n_chunks = L.get().P * C;  // the chosen layout's chunks
    const int32_t o0 = goff[gr], o1 = goff[gr + 1];
    if (o0 == o1) {
        out[gr] = make_int2(-1, -1);
        return;
    }
    auto holding = [&](int32_t t) {  // last c in [0, n_chunks) with chunk_rec[c] <= t
        int lo = 0, hi = n_chunks;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (chunk_rec[mid] <= t) lo = mid; else hi = mid;
        }
        return lo;
    };
    out[gr] = make_int2(holding(o0), holding(o1 - 1));
}

// ---- power tables -----------------------------------------------------------
// y viewed as a matrix Y[P][S] (flat i = p S + s).  Element (p, s) yields
// z = (y - c) / s_scale and its powers z^j 2^e, j = 1..4 (FP64, then rounded).
// mode 0: out[(p*4 + j) * ld + s]      (rows (p, j), cols s)
// mode 1: out[s * ld + p*4 + j]        (rows s, cols (p, j))
// mode 2: out[(s*4 + j) * ld + p]      (rows (s, j), cols p)
// mode 3: out[p * ld + s*4 + j]        (rows p, cols (s, j))
// A 32 x 32 (p, s) tile goes through shared memory so that both the read of y
// and the write of the table are coalesced whatever the mode.
template <typename T>
struct Store;
template <>
struct Store<float> {
    static __device__ __forceinline__ void put(float *o, float * /*o2*/, int64_t idx, double v) {
        o[idx] = (float)v;
    }
};

// TF32 pair: hi = v rounded to TF32 (10 explicit mantissa bits, stored in a
// float), lo = the remainder rounded to TF32.
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
struct Tf32Pair {};
template <>
struct Store<Tf32Pair> {
    static __device__ __forceinline__ void put(float *o, float *o2, int64_t idx, double v) {
        const float h = to_tf32((float)v);
        o[idx] = h;
        o2[idx] = to_tf32((float)(v - (double)h));
    }
};

template <typename T, typename O = T>
__global__ void k_power_table(const double *__restrict__ y, int64_t P, int64_t S,
                              const double *__restrict__ sc, int mode, int64_t ld,
                              O *__restrict__ out, O *__restrict__ out2) {
    __shared__ double tile[32][33];
    const int64_t p0 = (int64_t)blockIdx.y * 32, s0 = (int64_t)blockIdx.x * 32;
    const double scale = sc[kScaleS], shift = sc[kScaleC], pf = sc[kScaleP];
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int64_t p = p0 + r, s = s0 + threadIdx.x;
        double z = 0.0;
        if (p < P && s < S) z = __ddiv_rn(__dsub_rn(y[p * S + s], shift), scale);
        tile[r][threadIdx.x] = z;
    }
    __syncthreads();
    // 32 x 32 x 4 values; thread t handles values linear in the output order
    const int tid = threadIdx.y * 32 + threadIdx.x, nthr = 32 * blockDim.y;
    for (int e = tid; e < 32 * 32 * 4; e += nthr) {
        int a, b, j;  // a = fast output coordinate within the tile
        int lp, ls;
        int64_t idx;
        switch (mode) {
        case 0: {  // rows (p, j), cols s : fast = s
            ls = e & 31; j = (e >> 5) & 3; lp = e >> 7;
            idx = ((p0 + lp) * 4 + j) * ld + (s0 + ls);
            break;
        }
        case 1: {  // rows s, cols (p, j) : fast = (p, j)
            j = e & 3; lp = (e >> 2) & 31; ls = e >> 7;
            idx = (s0 + ls) * ld + (p0 + lp) * 4 + j;
            break;
        }
        case 2: {  // rows (s, j), cols p : fast = p
            lp = e & 31; j = (e >> 5) & 3; ls = e >> 7;
            idx = ((s0 + ls) * 4 + j) * ld + (p0 + lp);
            break;
        }
        default: {  // rows p, cols (s, j) : fast = (s, j)
            j = e & 3; ls = (e >> 2) & 31; lp = e >> 7;
            idx = (p0 + lp) * ld + (s0 + ls) * 4 + j;
            break;
        }
        }
        (void)a; (void)b;
        if (p0 + lp >= P || s0 + ls >= S) continue;
        double z = tile[lp][ls];
        double v = z;
        for (int q = 0; q < j; ++q) v = v * z;
        Store<T>::put(out, out2, idx, v * pf);
    }
}

// Split BF16 power table (the tensor-core B operand): z = (y - c) / s_scale,
// then z^j 2^e in FP32 (z 2^e, then times z: the power-of-two factor is exact
// and keeps the powers of small z normal) and the BF16 hi / lo split of each.  z comes from one FP64
// difference and product with 1 / s_scale rounded once to FP32 (within an
// FP32 ulp of the quotient), the powers carry at most three more FP32 roundings: far below
// the 2^-17 relative resolution of the hi + lo pair.  FP64 stays on the
// per-element path only for that one product (FP64 is the slow pipe here).
// Modes 0 and 2 of k_power_table.
// Split BF16 power table of the tensor-core contraction, [rest * 4 + j][red]
// with row stride ld: element (rest, red) of y (y[rest * Rn + red] when
// REST_ROWS, else y[red * Qn + rest]) yields z = (y - c) / s_scale and z^(j+1),
// j = 0..3, each split into BF16 hi + lo.  The grid covers the padded table
// (rests up to Qext, reds up to ld, both multiples of 64) and writes zeros
// there.  A 32 (rest) x 64 (red) tile of z goes through shared memory; each
// thread stores two consecutive reds (4 bytes) per row.
template <bool REST_ROWS>
__global__ void k_power_table_bf16(const double *__restrict__ y, int64_t Qn, int64_t Rn, int64_t Qext,
                                   const double *__restrict__ sc, int64_t ld, __nv_bfloat16 *__restrict__ out,
                                   __nv_bfloat16 *__restrict__ out2) {
    pdl_trigger();
    pdl_wait();
    __shared__ float tile[32][65];
    const int64_t q0 = (int64_t)blockIdx.y * 32, r0 = (int64_t)blockIdx.x * 64;
    const double inv = 1.0 / sc[kScaleS], shift = sc[kScaleC];
    const float pf = (float)sc[kScaleP];
    for (int e = threadIdx.x; e < 32 * 64; e += blockDim.x) {
        int lq, lr;
        if (REST_ROWS) {
            lq = e >> 6;
            lr = e & 63;
        } else {
            lq = e & 31;
            lr = e >> 5;
        }
        const int64_t q = q0 + lq, r = r0 + lr;
        float z = 0.f;
        if (q < Qn && r < Rn) z = (float)__dmul_rn(__dsub_rn(y[REST_ROWS ? q * Rn + r : r * Qn + q], shift), inv);
        tile[lq][lr] = z;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 4 * 32; e += blockDim.x) {
        const int pr = e & 31, j = (e >> 5) & 3, lq = e >> 7;
        const int64_t q = q0 + lq, r = r0 + 2 * pr;
        if (q >= Qext) continue;
        const float z0 = tile[lq][2 * pr], z1 = tile[lq][2 * pr + 1];
        float v0 = z0 * pf, v1 = z1 * pf;
        for (int t = 0; t < j; ++t) {
            v0 *= z0;
            v1 *= z1;
        }
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
        const int64_t idx = (q * 4 + j) * ld + r;
        *reinterpret_cast<__nv_bfloat162 *>(out + idx) = __halves2bfloat162(h0, h1);
        *reinterpret_cast<__nv_bfloat162 *>(out2 + idx) = __halves2bfloat162(
            __float2bfloat16_rn(v0 - __bfloat162float(h0)), __float2bfloat16_rn(v1 - __bfloat162float(h1)));
    }
}

}  // namespace

// ---------------------------------------------------------------- host side
// Exclusive scan of L int32 values; `scratch` holds the per-level block sums
// (scan_scratch_ints(L) entries).
static int64_t scan_scratch_ints(int64_t L) {
    int64_t total = 0;
    for (int64_t nb = ceil_div64(L, kScanBlock); nb > 1; nb = ceil_div64(nb, kScanBlock))
        total += 2 * nb + 64;
    return total + 64;
}

// Kernel launches of scan_exclusive over L elements.
static int scan_launches(int64_t L) {
    const int64_t nb = ceil_div64(L, kScanBlock);
    return nb <= 1 ? 1 : 2 + scan_launches(nb);
}

// (T = int32_t or unsigned long long; scratch counted in T elements)
template <typename T>
static vup_status scan_exclusive(const T *in, T *out, int64_t L, T *scratch, cudaStream_t s,
                                 const int32_t *gate = nullptr) {
    const int64_t nb = ceil_div64(L, kScanBlock);
    if (nb <= 1) {
        k_scan_blocks<T><<<1, kScanThreads, 0, s>>>(in, out, L, nullptr, gate);
        VUP_CHECK_LAUNCH();
        return VUP_OK;
    }
    T *sums = scratch;
    T *sums_scan = scratch + nb + 32;
    k_scan_blocks<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, L, sums, gate);
    VUP_CHECK_LAUNCH();
    vup_status st = scan_exclusive<T>(sums, sums_scan, nb, scratch + 2 * nb + 64, s, gate);
    if (st != VUP_OK) return st;
    k_scan_add<T><<<(unsigned)nb, 256, 0, s>>>(out, L, sums_scan, gate);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}

static GridGeom geom_of(vup_grid g) {
    GridGeom G;
    G.ndim = g->ndim;
    for (int d = 0; d < 3; ++d) {
        G.n[d] = g->n[d];
        G.lo[d] = g->lo[d];
        G.h[d] = (g->hi[d] - g->lo[d]) / (double)g->n[d];
    }
    return G;
}

// The built-in model at K arbitrary points x [K][ndim] (same arithmetic as
// the grid evaluation).
__global__ void k_model_at(const double *__restrict__ x, int64_t K, int ndim, int model, Theta th,
                           double *__restrict__ y) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= K) return;
    double p[3] = {0, 0, 0};
    for (int d = 0; d < ndim; ++d) p[d] = x[k * ndim + d];
    y[k] = model_value(model, th, p, ndim);
}

vup_status vup_launch_model_at(vup_grid g, int64_t K, const double *x, double *y, cudaStream_t s) {
    Theta th;
    for (int q = 0; q < 8; ++q) th.t[q] = g->theta[q];
    VUP_PROF("model_at", s, 1);
    k_model_at<<<(unsigned)ceil_div64(K, 128), 128, 0, s>>>(x, K, g->ndim, g->model_id, th, y);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}

vup_status vup_launch_model_eval(vup_grid g, int model_id, const double *theta, cudaStream_t s) {
    Theta th;
    for (int q = 0; q < 8; ++q) th.t[q] = theta[q];
    GridGeom G = geom_of(g);
    int blocks = (int)std::min<int64_t>(ceil_div64(g->N, 256), (int64_t)vup_num_sms() * 8);
    const bool sep = model_separable(model_id, g->ndim);
    VUP_PROF("model_eval", s, sep ? 2 : 1);
    VUP_CHECK_CUDA(cudaMemsetAsync(g->ext, 0xff, sizeof(unsigned long long), s));
    VUP_CHECK_CUDA(cudaMemsetAsync(g->ext + 1, 0x00, 2 * sizeof(unsigned long long), s));
    g->bins_ready = 0;
    if (sep) {
        int64_t nmax = 1;
        for (int d = 0; d < g->ndim; ++d) nmax = std::max(nmax, g->n[d]);
        VUP_CHECK_CUDA(launch_pdl(k_axis_terms, dim3((unsigned)ceil_div64(nmax, 128)), dim3(128), 0, s, G, model_id, th,
                                  g->axis_terms));
        VUP_CHECK_LAUNCH();
        if (g->ndim >= 2) {
            // values, range and bins in one cooperative launch (every block resident)
            static int per_sm = 0;
            if (!per_sm) VUP_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_model_bins, 256, 0));
            const int cb = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div64(g->N, 256),
                                                                        (int64_t)vup_num_sms() * std::max(1, per_sm)));
            double *y = g->y;
            int64_t N = g->N;
            const double2 *terms = (const double2 *)g->axis_terms;
            unsigned long long *ext = g->ext;
            int B = g->B;
            int32_t *bins = g->bins;
            double *sc = g->ydev_scale;
            int *dstatus = g->dstatus;
            int mid = model_id;
            // the tensor-core orientation's split BF16 power table as well
            // (built here for the default precision; kept until the next model)
            const int to = vup_tc_orient(g);
            const Orient &o = g->orient[to];
            int64_t ld = o.R_pad, R = o.R, Qext = ceil_div64(o.NC, 256) * 256 / 4;
            const size_t tbytes = sizeof(__nv_bfloat16) * (size_t)ld * (size_t)(Qext * 4);
            if (!g->zt_hi[to]) {
                VUP_CHECK_CUDA(vup_dev_malloc(&g->zt_hi[to], tbytes));
                VUP_CHECK_CUDA(vup_dev_malloc(&g->zt_lo[to], tbytes));
            }
            __nv_bfloat16 *zh = g->zt_hi[to], *zl = g->zt_lo[to];
            void *args[] = {&y, &N, &G, &mid, &th, &terms, &ext, &B, &bins, &sc, &dstatus, &zh, &zl, &R, &ld, &Qext};
            VUP_CHECK_CUDA(cudaLaunchCooperativeKernel((const void *)k_model_bins, dim3(cb), dim3(256), args, 0, s));
            g->bins_ready = 1;
        } else {
            VUP_CHECK_CUDA(launch_pdl(k_model_combine, dim3(blocks), dim3(256), 0, s, g->y, g->N, G, model_id, th,
                                      (const double2 *)g->axis_terms, g->ext));
        }
    } else {
        k_model_eval<<<blocks, 256, 0, s>>>(g->y, g->N, G, model_id, th, g->ext);
    }
    g->range_ready = 1;
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}

int vup_hist_chunks_for(int64_t N, int P);
int vup_hist_parts_for(int64_t n_last, int n_bins);

// Warps per CTA of the counting-sort kernels for a key space of Bk keys (the
// per-warp counters of Bk ints must fit 128 KB of shared memory).
static int sort_warps(int Bk) { return std::max(1, std::min(kSortWarps, 32768 / std::max(Bk, 1))); }

// Stable counting sort of `keys` (values < Bk) into perm; key offsets to koff
// (Bk + 1 entries) when koff is not null.  `counts` must hold 2 Bk n_tiles + 8.
static vup_status counting_sort(vup_grid g, const int32_t *keys, int Bk, int32_t *perm, int32_t *koff,
                                int32_t *counts, int32_t *scratch, bool counts_ready, cudaStream_t s,
                                const int32_t *gate = nullptr) {
    const int64_t N = g->N;
    const int64_t n_tiles = ceil_div64(N, kSortTile);
    const int64_t L = (int64_t)Bk * n_tiles;
    int32_t *starts = counts + L + 4;
    const int nw = sort_warps(Bk);
    const size_t smem = sizeof(int32_t) * (size_t)Bk * nw;
    const unsigned blocks = (unsigned)ceil_div64(n_tiles, nw);
    if (smem > 48 * 1024) {
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        VUP_CHECK_CUDA(cudaFuncSetAttribute(k_sort_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (!counts_ready) {
        k_count<<<blocks, 32 * nw, smem, s>>>(keys, N, Bk, counts, n_tiles, gate);
        VUP_CHECK_LAUNCH();
    }
    vup_status st = scan_exclusive(counts, starts, L, scratch, s, gate);
    if (st != VUP_OK) return st;
    k_sort_scatter<<<blocks, 32 * nw, smem, s>>>(keys, N, Bk, gate, starts, n_tiles, perm);
    VUP_CHECK_LAUNCH();
    if (koff) {
        k_koff<<<(Bk + 1 + 255) / 256, 256, 0, s>>>(starts, n_tiles, Bk, N, koff, gate);
        VUP_CHECK_LAUNCH();
    }
    return VUP_OK;
}

// The CSR form of the one-hot model matrix (points stably sorted by bin) for
// grids whose histogram runs on a layout stream; built when first asked for.
vup_status vup_natural_sort(vup_grid g, cudaStream_t s) {
    if (g->natural_valid) return VUP_OK;
    int32_t *scratch = (int32_t *)g->scan_tmp.p;
    vup_status st = counting_sort(g, g->bins, g->B, g->perm, g->offsets, (int32_t *)g->sort_counts.p, scratch, false, s);
    if (st != VUP_OK) return st;
    g->natural_valid = 1;
    return VUP_OK;
}

vup_status vup_launch_grid_finish(vup_grid g, cudaStream_t s) {
    const int64_t N = g->N;
    const int B = g->B;
    ProfScope prof("range_bins", s, 0);
    const bool bins_done = g->bins_ready && g->range_ready;  // the model kernel wrote them
    g->bins_ready = 0;
    int launches = g->ndim == 1 ? 2 : (bins_done ? 0 : 1);  // scale, bins
    // exact range of y (already reduced by the model kernels for built-in models)
    int blocks = (int)std::min<int64_t>(ceil_div64(N, 256), (int64_t)vup_num_sms() * 8);
    if (!g->range_ready) {
        VUP_CHECK_CUDA(cudaMemsetAsync(g->ext, 0xff, sizeof(unsigned long long), s));
        VUP_CHECK_CUDA(cudaMemsetAsync(g->ext + 1, 0x00, sizeof(unsigned long long), s));
        k_minmax<<<blocks, 256, 0, s>>>(g->y, N, g->ext);
        VUP_CHECK_LAUNCH();
        ++launches;
    }
    g->range_ready = 0;
    if (g->ndim == 1) {
        k_scale<<<1, 1, 0, s>>>(g->ext, N, g->ydev_scale);
        VUP_CHECK_LAUNCH();
    }

    // parts of each candidate layout's gathered axis for this bin count; the
    // arrays of the one layout that is built live in hl[0] (hl[1] aliases them)
    int Bk_max = B;
    g->hist_P = 1;
    if (g->ndim >= 2) {
        for (int l = 0; l < g->n_layouts; ++l) {
            auto &HL = g->hl[l];
            HL.P = vup_hist_parts_for(HL.n_last, B);
            HL.part_rows = ceil_div64(HL.n_last, HL.P);
            Bk_max = std::max(Bk_max, HL.P * B);
            g->hist_P = std::max(g->hist_P, HL.P);
        }
        auto &HL = g->hl[0];
        if (HL.koff_cap < Bk_max + 1) {
            cudaFree(HL.koff);
            cudaFree(HL.key_chunks);
            HL.koff = nullptr;
            HL.key_chunks = nullptr;
            VUP_CHECK_CUDA(vup_dev_malloc(&HL.koff, sizeof(int32_t) * (Bk_max + 1)));
            VUP_CHECK_CUDA(vup_dev_malloc(&HL.key_chunks, sizeof(int2) * (Bk_max + 1)));
            HL.koff_cap = Bk_max + 1;
        }
        if (g->n_layouts > 1) {
            g->hl[1].koff = HL.koff;
            g->hl[1].key_chunks = HL.key_chunks;
            g->hl[1].koff_cap = HL.koff_cap;
        }
    }
    const int64_t n_tiles = ceil_div64(N, kSortTile);
    const int64_t Lmax = (int64_t)Bk_max * n_tiles;
    vup_status st = devbuf_reserve(g->sort_counts, sizeof(int32_t) * (size_t)std::max<int64_t>(2 * Lmax + 8, N + 8));
    if (st != VUP_OK) return st;
    st = devbuf_reserve(g->scan_tmp, sizeof(unsigned long long) *
                                         (size_t)scan_scratch_ints(std::max<int64_t>(Lmax, N)));
    if (st != VUP_OK) return st;
    int32_t *scratch = (int32_t *)g->scan_tmp.p;
    int32_t *counts = (int32_t *)g->sort_counts.p;

    // bins (Eq. 4), counted per tile for the sort by bin
    {
        if (g->ndim == 1) {
            const int nw = sort_warps(B);
            const size_t smem = sizeof(int32_t) * (size_t)B * nw;
            if (smem > 48 * 1024)
                VUP_CHECK_CUDA(
                    cudaFuncSetAttribute(k_bins_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_bins_count<<<(unsigned)ceil_div64(n_tiles, nw), 32 * nw, smem, s>>>(g->y, N, B, g->ext, g->bins,
                                                                                counts, n_tiles);
        } else if (!bins_done) {
            const int bb = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div64(N / 2, 256), (int64_t)vup_num_sms() * 8));
            VUP_CHECK_CUDA(launch_pdl(k_bins_scale, dim3(bb), dim3(256), 0, s, (const double *)g->y, N, B,
                                      (const unsigned long long *)g->ext, g->bins, g->ydev_scale));
        }
        VUP_CHECK_LAUNCH();
    }
    g->natural_valid = 0;
    if (g->ndim == 1) {
        // the 1-D path walks the model matrix in CSR form directly
        st = counting_sort(g, g->bins, B, g->perm, g->offsets, counts, scratch, true, s);
        if (st != VUP_OK) return st;
        g->natural_valid = 1;
        launches += 2 + scan_launches((int64_t)B * n_tiles);
    }
    g->layout_valid = g->ndim == 1;
    prof.launches = launches;
    for (int o = 0; o < kNumOrient; ++o) g->have_tab[o][0] = g->have_tab[o][1] = g->have_tab[o][2] = 0;
    if (bins_done) g->have_tab[vup_tc_orient(g)][1] = 1;  // written with the bins
    return VUP_OK;
}

// The histogram layout of a 2-D / 3-D grid (sorted point and interval
// streams, chunks, the natural bin offsets) for the current bins.  Built on
// first use after a model evaluation (the histogram, the bin offsets), so a
// caller may run it on a second stream beside the density preparation.
vup_status vup_build_layout(vup_grid g, cudaStream_t s, bool points_needed, cudaEvent_t records_done,
                            cudaEvent_t layout_picked) {
    const int64_t N = g->N;
    const int B = g->B;
    // two timed parts: up to the record-stream decision, and the key-sorted streams
    std::unique_ptr<ProfScope> prof_rec(new ProfScope("layout_sort_records", s, 0));
    int launches = 0;
    int Bk_max = B;
    for (int l = 0; l < g->n_layouts; ++l) Bk_max = std::max(Bk_max, g->hl[l].P * B);
    const int64_t n_tiles = ceil_div64(N, kSortTile);
    int32_t *scratch = (int32_t *)g->scan_tmp.p;
    int32_t *counts = (int32_t *)g->sort_counts.p;
    const int blocks = (int)std::min<int64_t>(ceil_div64(N, 256), (int64_t)vup_num_sms() * 8);
    vup_status st;
    {
        const int C = g->n_chunks;
        auto &HL = g->hl[0];
        LaySel L;
        for (int l = 0; l < 2; ++l) {
            const auto &h = g->hl[l < g->n_layouts ? l : 0];
            L.g[l] = LayGeom{h.n_last, h.part_rows, h.P};
        }
        L.sel = g->hist_sel;
        int32_t *iv_cnt = g->hist_sel + 2;
        if (g->n_layouts > 1) {
            // the layout with fewer intervals (counted without sorting)
            VUP_CHECK_CUDA(cudaMemsetAsync(iv_cnt, 0, 2 * sizeof(int32_t), s));
            k_iv_count<<<blocks, 256, 0, s>>>(g->bins, g->n[0], g->n[1], B, L, iv_cnt);
            VUP_CHECK_LAUNCH();
            k_pick_layout<<<1, 1, 0, s>>>(iv_cnt, g->hist_sel);
            VUP_CHECK_LAUNCH();
            launches += 2;
        }
        if (layout_picked) VUP_CHECK_CUDA(cudaEventRecord(layout_picked, s));
        const int rb = (int)std::min<int64_t>(ceil_div64(N, 256), (int64_t)vup_num_sms() * 8);
        const int64_t Cn = HL.n_last, Rn = N / Cn;  // bins as [R][C], C = the last axis
        // record stream, walked line by line from the bins
        {
            const int GB = (int)ceil_div64(B, kRecBins);
            int P_sel = 1;
            int64_t NL = 1, walkers = 1;
            for (int l = 0; l < g->n_layouts; ++l) {
                const int64_t lines = l == 0 ? Rn : Cn;
                P_sel = std::max(P_sel, g->hl[l].P);
                NL = std::max(NL, lines);
                walkers = std::max(walkers, (int64_t)g->hl[l].P * lines);
            }
            const int n_groups = P_sel * GB;  // room for either layout's parts
            const int64_t Lr = (int64_t)n_groups * NL;
            int64_t cap = 1;
            for (int l = 0; l < g->n_layouts; ++l) cap = std::max(cap, g->hl[l].part_rows);
            // counts, their scan, segment record counts, then the uint4 slots (16-byte aligned)
            const int64_t ints = ((2 * Lr + walkers + 3) / 4) * 4;
            if ((st = devbuf_reserve(g->rec_tmp, sizeof(int32_t) * (size_t)ints +
                                                     sizeof(uint4) * 2 * (size_t)(walkers * cap))) != VUP_OK ||
                (st = devbuf_reserve(g->scan_tmp, sizeof(unsigned long long) * (size_t)scan_scratch_ints(Lr))) !=
                    VUP_OK ||
                (st = devbuf_reserve(HL.rec, sizeof(uint4) * 2 * (size_t)(N + 64))) != VUP_OK ||
                (st = devbuf_reserve(HL.rec_rest, sizeof(int32_t) * (size_t)(N + 64))) != VUP_OK ||
                (st = devbuf_reserve(HL.rec_goff, sizeof(int32_t) * (size_t)(n_groups + 2))) != VUP_OK ||
                (st = devbuf_reserve(HL.rec_gch, sizeof(int2) * (size_t)n_groups)) != VUP_OK)
                return st;
            scratch = (int32_t *)g->scan_tmp.p;
            int32_t *rcnt = (int32_t *)g->rec_tmp.p, *rstart = rcnt + Lr, *seg_n = rcnt + 2 * Lr;
            uint4 *rslot = reinterpret_cast<uint4 *>(rcnt + ints);
            RecGeom Q;
            Q.R = Rn;
            Q.C = Cn;
            Q.GB = GB;
            Q.NL = NL;
            Q.cap = cap;
            Q.ndim = g->ndim;
            Q.n1 = g->ndim == 3 ? g->n[1] : 1;
            VUP_CHECK_CUDA(cudaMemsetAsync(rcnt, 0, sizeof(int32_t) * (size_t)Lr, s));
            VUP_CHECK_CUDA(cudaMemsetAsync(HL.n_iv, 0, sizeof(int32_t), s));
            const size_t wsm = sizeof(int32_t) * (size_t)kWalkWarps * GB;
            if (wsm > 48 * 1024)
                VUP_CHECK_CUDA(cudaFuncSetAttribute(k_rec_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm));
            k_rec_walk<<<(unsigned)ceil_div64(walkers, kWalkWarps), kWalkWarps * 32, wsm, s>>>(g->bins, Q, L, rcnt,
                                                                                             HL.n_iv, rslot, seg_n);
            VUP_CHECK_LAUNCH();
            if ((st = scan_exclusive(rcnt, rstart, Lr, scratch, s)) != VUP_OK) return st;
            k_rec_goff<<<(n_groups + 2 + 255) / 256, 256, 0, s>>>(rstart, rcnt, Lr, NL, n_groups,
                                                                  (int32_t *)HL.rec_goff.p, HL.n_rec);
            VUP_CHECK_LAUNCH();
            k_rec_scatter<<<(unsigned)std::min<int64_t>(ceil_div64(walkers, 8), (int64_t)vup_num_sms() * 16), 256, 0,
                            s>>>(rslot, seg_n, Q, L, rstart, (const int32_t *)HL.rec_goff.p, HL.n_rec,
                                 (uint4 *)HL.rec.p, (int32_t *)HL.rec_rest.p);
            VUP_CHECK_LAUNCH();
            // chunks of records (the same count per part as the other streams' chunks / 4)
            const int Cr = g->n_chunks_rec;
            k_rec_chunks<<<(P_sel * Cr + 1 + 127) / 128, 128, 0, s>>>((const int32_t *)HL.rec_goff.p, HL.n_rec, GB, L,
                                                                      Cr, (const uint4 *)HL.rec.p, HL.rec_chunk,
                                                                      HL.rec_chunk_grp);
            VUP_CHECK_LAUNCH();
            k_rec_group_chunks<<<(n_groups + 127) / 128, 128, 0, s>>>((const int32_t *)HL.rec_goff.p, n_groups,
                                                                       HL.rec_chunk, L, Cr,
                                                                       (int2 *)HL.rec_gch.p);
            VUP_CHECK_LAUNCH();
            // walk, scan, first records, scatter, chunks, group chunks, gate
            launches += 2 + scan_launches(Lr) + 2 + 2 + 1;
        }
        // the key-sorted point and interval streams, unless the record stream is
        // cheaper than both (every kernel below then returns at once); the
        // point stream is always built for callers that walk it -- posterior
        // means -- and where the shared-memory kernels cannot run
        const int32_t *gate = g->hist_sel + 4;
        const bool force_keys = points_needed || !vup_hist_tile_fits(g);
        k_need_keys<<<1, 1, 0, s>>>(HL.n_rec, HL.n_iv, N, g->ndim - 1, g->hist_force, force_keys ? 1 : 0,
                                    g->hist_sel, HL.n_runs);
        VUP_CHECK_LAUNCH();
        // a caller may start the record-stream histogram from here on
        prof_rec->launches = launches;
        prof_rec.reset();
        launches = 0;
        if (records_done) VUP_CHECK_CUDA(cudaEventRecord(records_done, s));
        ProfScope prof("layout_sort_runs", s, 0);
        // sort keys of the chosen layout in its order, stable counting sort
        dim3 tg((unsigned)ceil_div64(Cn, 32), (unsigned)std::min<int64_t>(ceil_div64(Rn, 32), 65535));
        k_layout_keys<<<tg, dim3(32, 8), 0, s>>>(g->bins, Rn, Cn, B, L, HL.keys_own, gate);
        VUP_CHECK_LAUNCH();
        HL.keys = HL.keys_own;
        st = counting_sort(g, HL.keys, Bk_max, HL.perm, HL.koff, counts, scratch, false, s, gate);
        if (st != VUP_OK) return st;
        // runs and intervals: one flag word per point, one 64-bit scan
        st = devbuf_reserve(g->lay_tmp, sizeof(unsigned long long) * 2 * (size_t)N);
        if (st != VUP_OK) return st;
        auto *flags = (unsigned long long *)g->lay_tmp.p;
        auto *excl = flags + N;
        k_layout_flags<<<rb, 256, 0, s>>>(HL.perm, HL.keys, N, L, flags, gate);
        VUP_CHECK_LAUNCH();
        st = scan_exclusive<unsigned long long>(flags, excl, N, (unsigned long long *)g->scan_tmp.p, s, gate);
        if (st != VUP_OK) return st;
        k_layout_build<<<rb, 256, 0, s>>>(HL.perm, HL.keys, N, L, kRowShift, flags, excl, HL.run_start, HL.run_rest,
                                          HL.run_bin, HL.hpt, HL.n_runs, HL.ipt, HL.iv_rest, HL.n_iv, gate);
        VUP_CHECK_LAUNCH();
        // run-end words carry the rest code of the run kRunAhead places later
        // (their factors come from L2, loaded that far ahead), or of the next
        // run when the 3-D point stream stages the rest factors in shared memory
        const int run_ahead = vup_hist_rest_staged(g) ? 1 : kRunAhead;
        k_layout_encode<<<rb, 256, 0, s>>>(HL.run_start, HL.run_rest, HL.n_runs, HL.iv_rest, HL.n_iv, g->ndim,
                                           g->ndim == 3 ? g->n[1] : 1, kRowShift, HL.hpt, HL.ipt, run_ahead, gate);
        VUP_CHECK_LAUNCH();
        // chunks of every part
        const int PC = g->hist_P * C;
        k_chunks<<<(PC + 1 + 127) / 128, 128, 0, s>>>(HL.run_start, HL.n_runs, HL.koff, B, L, C, excl, N, HL.n_iv,
                                                       HL.chunk_pt, HL.chunk_run, HL.chunk_iv, gate);
        VUP_CHECK_LAUNCH();
        k_chunk_bins<<<(PC + 127) / 128, 128, 0, s>>>(HL.chunk_run, HL.run_bin, L, C, HL.chunk_bin, gate);
        VUP_CHECK_LAUNCH();
        k_key_chunks<<<(Bk_max + 127) / 128, 128, 0, s>>>(HL.koff, L, B, HL.chunk_pt, C, HL.key_chunks, gate);
        VUP_CHECK_LAUNCH();
        st = vup_pick_hist_layout(g, s);
        if (st != VUP_OK) return st;
        // keys, sort (count, scan, scatter, koff end), flags, scan, build, encode, chunks,
        // chunk keys, key chunks, stream choice
        launches += 1 + 3 + scan_launches((int64_t)Bk_max * n_tiles) + 1 + scan_launches(N) + 2 + 4;
        prof.launches = launches;
    }
    g->layout_valid = 1;
    g->layout_has_points = points_needed || g->ndim == 1;
    return VUP_OK;
}

vup_status vup_ensure_layout(vup_grid g, cudaStream_t s, bool points_needed) {
    if (g->layout_valid && (!points_needed || g->layout_has_points)) return VUP_OK;
    return vup_build_layout(g, s, points_needed);
}

vup_status vup_pick_hist_layout(vup_grid g, cudaStream_t s) {
    k_pick_stream<<<1, 1, 0, s>>>(g->hl[0].n_runs, g->hl[0].n_iv, g->N, g->hist_force, g->hist_sel);
    VUP_CHECK_LAUNCH();
    return VUP_OK;
}

// Build (lazily) the power tables of orientation `orient` in FP32 (SIMT
// layout [R][NC]) or split BF16 (tensor layout [NC][R_pad]).
vup_status vup_build_tables(vup_grid g, int orient, int bf16, cudaStream_t s) {
    if (g->have_tab[orient][bf16]) return VUP_OK;
    // bf16: 0 = FP32 (SIMT layout), 1 = BF16 hi/lo, 2 = TF32 hi/lo (tensor layouts)
    const Orient &o = g->orient[orient];
    // View y as [P][S]: orientations 0 and 2 -> P = rest (Q), S = red (R)
    // (the reduction axes are the trailing ones); orientation 1 (2-D) ->
    // P = axis 0 = red, S = axis 1 = rest.
    const bool first = orient == kOrientFirst;
    const int64_t P = first ? o.R : o.Q;
    const int64_t S = first ? o.Q : o.R;
    dim3 blk(32, 8), grd((unsigned)ceil_div64(S, 32), (unsigned)ceil_div64(P, 32));
    VUP_PROF(bf16 == 2 ? "power_table_tf32" : (bf16 ? "power_table_bf16" : "power_table_fp32"), s, 1);
    if (!bf16) {
        const int64_t ld = ceil_div64(o.NC, 128) * 128;
        const size_t bytes = sizeof(float) * (size_t)ld * (size_t)o.R;
        if (!g->zs[orient]) VUP_CHECK_CUDA(vup_dev_malloc(&g->zs[orient], bytes));
        VUP_CHECK_CUDA(cudaMemsetAsync(g->zs[orient], 0, bytes, s));
        // SIMT wants [r][q*4+j]: orientation 0 -> rows s (mode 1); 1 -> rows p (mode 3)
        k_power_table<float><<<grd, blk, 0, s>>>(g->y, P, S, g->ydev_scale, first ? 3 : 1, ld,
                                                 g->zs[orient], (float *)nullptr);
        VUP_CHECK_LAUNCH();
    } else if (bf16 == 2) {
        const int64_t ld = o.R_pad;
        const int64_t rows = ceil_div64(o.NC, 256) * 256;
        const size_t bytes = sizeof(float) * (size_t)ld * (size_t)rows;
        if (!g->ztf_hi[orient]) {
            VUP_CHECK_CUDA(vup_dev_malloc(&g->ztf_hi[orient], bytes));
            VUP_CHECK_CUDA(vup_dev_malloc(&g->ztf_lo[orient], bytes));
        }
        VUP_CHECK_CUDA(cudaMemsetAsync(g->ztf_hi[orient], 0, bytes, s));
        VUP_CHECK_CUDA(cudaMemsetAsync(g->ztf_lo[orient], 0, bytes, s));
        k_power_table<Tf32Pair, float><<<grd, blk, 0, s>>>(g->y, P, S, g->ydev_scale, first ? 2 : 0, ld,
                                                          g->ztf_hi[orient], g->ztf_lo[orient]);
        VUP_CHECK_LAUNCH();
    } else {
        const int64_t ld = o.R_pad;
        const int64_t rows = ceil_div64(o.NC, 256) * 256;
        const size_t bytes = sizeof(__nv_bfloat16) * (size_t)ld * (size_t)rows;
        if (!g->zt_hi[orient]) {
            VUP_CHECK_CUDA(vup_dev_malloc(&g->zt_hi[orient], bytes));
            VUP_CHECK_CUDA(vup_dev_malloc(&g->zt_lo[orient], bytes));
        }
        // tensor wants [q*4+j][r], padding included: y is [Q][R] (orientations 0
        // and 2) or [R][Q] (orientation 1)
        const int64_t Qext = rows / 4;
        dim3 pg((unsigned)(ld / 64), (unsigned)(Qext / 32));
        if (first)
            VUP_CHECK_CUDA(launch_pdl(k_power_table_bf16<false>, pg, dim3(256), 0, s, (const double *)g->y, o.Q, o.R,
                                      Qext, (const double *)g->ydev_scale, ld, g->zt_hi[orient], g->zt_lo[orient]));
        else
            VUP_CHECK_CUDA(launch_pdl(k_power_table_bf16<true>, pg, dim3(256), 0, s, (const double *)g->y, o.Q, o.R,
                                      Qext, (const double *)g->ydev_scale, ld, g->zt_hi[orient], g->zt_lo[orient]));
    }
    g->have_tab[orient][bf16] = 1;
    return VUP_OK;
}
