// Tensor-core (tcgen05 + TMA, sm_103a) form of the s = 2 elimination step
// (Appendix D: summing out an index with two live neighbours is the product
// C(j, k) = sum_i A(i, j) u(i) B(i, k)).  The product is stored, reduced in the
// epilogue against up to four weights (sum_jk C^p W a(j) b(k), p in {1, 2}), or
// both, so products consumed only by reductions never reach global memory.
//
// Split-bf16 modes.  Each K-major operand row X(j, .) is written as S bf16
// fixed-point slices relative to a power-of-two row scale s_j >= max |X(j, .)|:
//     X(j, i) = s_j 2^-w (d1 + d2 2^-8 + d3 2^-16 [+ d4 2^-24]),
//     d1 in [-2^w, 2^w], |d2|, |d3|, |d4| <= 128,
// every slice exact in bf16.  The product of two rows is accumulated as
//     ACC_hi = sum_i d1_A d1_B                   (integers: exact in FP32 because
//                                                 n 4^w <= 2^24)
//     ACC_lo = sum_i (all slice pairs of weight 2^-8 .. 2^-8(S-1))
// and C = s_j s_k 2^-2w (ACC_hi + ACC_lo).  S = 3 (6 products) or S = 4 (10
// products; 8 more bits for data whose rows span a wide dynamic range).  Exact
// accumulation of the leading term removes the rounding bias of the FP32
// accumulator, which would not average out over the n^2 terms of a V-statistic.
// TF32 mode: one tf32 copy of each operand (rounded to nearest), one accumulator.
//
// Kernel: persistent CTAs (one per SM), 192 threads.  Warp 0 streams A and B
// tiles with TMA into a ring of shared-memory stages (128-byte swizzle), warp 1
// issues tcgen05.mma (cta_group::1, M = 128, N = 128 or 64) into one of two TMEM
// accumulator buffers, warps 2-5 drain the other buffer (tcgen05.ld) in the
// epilogue, so the epilogue of one tile overlaps the main loop of the next.
// With `symmetric` (C = C^T and every reduction symmetric) only tiles on or
// above the diagonal are computed and off-diagonal tiles count twice.  Every
// mbarrier wait is bounded: on time-out the CTA records an error, waits (again
// bounded) for its MMAs and copies in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <type_traits>
#include <vector>
#include <cstdio>
#include <cstring>

#include "kcommon.cuh"
#include "kernels.h"
#include "kmath.cuh"
#include "tc_ptx.cuh"

namespace ustat {

int split_lead_bits(int64_t K) {
    int lg = 0;
    while ((int64_t(1) << lg) < K) ++lg;
    int w = (24 - lg) / 2;
    if (w > 8) w = 8;
    if (w < 1) w = 1;
    return w;
}

namespace {

// ------------------------------------------------------------------ split / prep

// Row-major source (X(j, i) = M[j][i] u(i)): one warp per operand row, two passes
// (row maximum, then digits), fully coalesced.
// With diag_out, a row whose diagonal entry X(j, j) sets a larger row scale than
// its other entries leaves the diagonal out (its digits 0, the row scale from the
// other entries) and writes its value to diag_out[j]; other rows keep it and
// write 0.  The GEMM epilogue adds the left-out terms exactly (diagonal
// correction).
template <typename T>
__global__ void __launch_bounds__(256) split_rows_kernel(const T *__restrict__ M, const double *__restrict__ u,
                                                         int64_t n, int64_t ldp, int lead_bits, int planes,
                                                         __nv_bfloat16 *__restrict__ slices,
                                                         float *__restrict__ scales, double *__restrict__ diag_out) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= n) return;
    const T *row = M + j * n;
    T mx = 0, moff = 0;
    if (std::is_same<T, double>::value && !u) {
        // float64 without weights: the maxima of |x| as integer maxima of the bit
        // patterns with the sign cleared (the same order for finite values)
        unsigned long long bm = 0, bo = 0;
        for (int64_t i = lane; i < n; i += 32) {
            const unsigned long long a = (unsigned long long)__double_as_longlong((double)row[i]) & 0x7FFFFFFFFFFFFFFFull;
            bm = a > bm ? a : bm;
            if (i != j) bo = a > bo ? a : bo;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long tm = __shfl_xor_sync(0xffffffffu, bm, o), to = __shfl_xor_sync(0xffffffffu, bo, o);
            bm = tm > bm ? tm : bm;
            bo = to > bo ? to : bo;
        }
        mx = (T)__longlong_as_double((long long)bm);
        moff = (T)__longlong_as_double((long long)bo);
    } else {
        for (int64_t i = lane; i < n; i += 32) {
            T x = row[i];
            if (u) x *= (T)u[i];
            mx = fmax(mx, fabs(x));
            if (i != j) moff = fmax(moff, fabs(x));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mx = (T)fmax((double)mx, (double)__shfl_xor_sync(0xffffffffu, mx, o));
            moff = (T)fmax((double)moff, (double)__shfl_xor_sync(0xffffffffu, moff, o));
        }
    }
    // leave the diagonal out whenever that lowers the row scale
    const bool drop = diag_out && row_exp(moff) < row_exp(mx);
    const int e = row_exp(drop ? moff : mx);
    if (lane == 0) scales[j] = ldexpf(1.f, e);
    const int64_t plane = n * ldp;
    for (int64_t i = lane; i < ldp; i += 32) {
        T x = 0;
        if (i < n) {
            x = row[i];
            if (u) x *= (T)u[i];
        }
        if (i == j) {
            if (diag_out) diag_out[j] = drop ? (double)x : 0.0;
            if (drop) x = 0;
        }
        write_digits(x, lead_bits, e, planes, slices + j * ldp + i, plane);
    }
}

// The value left out by skip_diag: out[j] = M[j][j] u(j), float64.
template <typename T>
__global__ void operand_diag_kernel(const T *__restrict__ M, const double *__restrict__ u, int64_t n,
                                    double *__restrict__ out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = (double)M[j * n + j] * (u ? u[j] : 1.0);
}

// s = 3 A operands from a row-major source: X_bb(j, i) = M[j][i] s_bb(i) with
// s_bb(i) = u(i) Ab(i, bb), Ab(i, bb) = transAb ? Mb[bb][i] : Mb[i][bb]; bb = bb0 +
// blockIdx.y.  s_bb is staged in shared memory once per block; one warp per
// operand row: the row maximum, then the digits of four consecutive entries per
// lane with 8-byte stores (the same digits as write_digits).
__global__ void __launch_bounds__(256) split_rows_g3_kernel(const float *__restrict__ M, const double *__restrict__ u,
                                                            const float *__restrict__ Mb, int transAb, int64_t bb0,
                                                            int64_t n, int64_t ldp, int lead_bits, int planes,
                                                            __nv_bfloat16 *__restrict__ slices,
                                                            float *__restrict__ scales) {
    extern __shared__ float sv[];   // [n]
    const int64_t bb = bb0 + blockIdx.y;
    slices += (int64_t)blockIdx.y * planes * n * ldp;
    scales += (int64_t)blockIdx.y * n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        float v = transAb ? Mb[bb * n + i] : Mb[i * n + bb];
        if (u) v *= (float)u[i];
        sv[i] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= n) return;
    const float *row = M + j * n;
    const bool vec = (n % 4) == 0;
    float mx = 0.f;
    for (int64_t i = 4 * lane; i < n; i += 128) {
        float x[4];
        if (vec) {
            const float4 r4 = *reinterpret_cast<const float4 *>(row + i);
            x[0] = r4.x, x[1] = r4.y, x[2] = r4.z, x[3] = r4.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = i + q < n ? row[i + q] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (i + q < n) mx = fmaxf(mx, fabsf(x[q] * sv[i + q]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = row_exp(mx);
    if (lane == 0) scales[j] = ldexpf(1.f, e);
    const int k = lead_bits - e;
    const bool pow2 = k >= -126 && k <= 127;
    const float p2 = pow2 ? __int_as_float((127 + k) << 23) : 0.f;
    const int64_t plane = n * ldp;
    for (int64_t i = 4 * lane; i < ldp; i += 128) {
        float y[4];
        if (vec && i + 3 < n) {
            const float4 r4 = *reinterpret_cast<const float4 *>(row + i);
            y[0] = r4.x * sv[i], y[1] = r4.y * sv[i + 1], y[2] = r4.z * sv[i + 2], y[3] = r4.w * sv[i + 3];
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) y[q] = i + q < n ? row[i + q] * sv[i + q] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) y[q] = pow2 ? y[q] * p2 : ldexpf(y[q], k);   // |y| <= 2^w, exact
        float d[4];
        float sc = 1.f;
        for (int p = 0; p < planes; ++p) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (p > 0) y[q] = (y[q] - d[q]) * 256.f;   // exact
                d[q] = rintf(y[q]);
            }
            const __nv_bfloat162 h01 = __floats2bfloat162_rn(d[0] * sc, d[1] * sc);
            const __nv_bfloat162 h23 = __floats2bfloat162_rn(d[2] * sc, d[3] * sc);
            *reinterpret_cast<uint2 *>(slices + p * plane + j * ldp + i) =
                make_uint2(*reinterpret_cast<const uint32_t *>(&h01), *reinterpret_cast<const uint32_t *>(&h23));
            sc *= (1.f / 256.f);
        }
    }
}

// The same for float64 sources (wide-storage mode): one warp per row, scalar.
__global__ void __launch_bounds__(256) split_rows_g3_wide_kernel(const double *__restrict__ M,
                                                                 const double *__restrict__ u,
                                                                 const double *__restrict__ Mb, int transAb,
                                                                 int64_t bb0, int64_t n, int64_t ldp, int lead_bits,
                                                                 int planes, __nv_bfloat16 *__restrict__ slices,
                                                                 float *__restrict__ scales) {
    const int64_t bb = bb0 + blockIdx.y;
    slices += (int64_t)blockIdx.y * planes * n * ldp;
    scales += (int64_t)blockIdx.y * n;
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= n) return;
    const double *row = M + j * n;
    auto val = [&](int64_t i) -> double {
        double x = row[i] * (transAb ? Mb[bb * n + i] : Mb[i * n + bb]);
        if (u) x *= u[i];
        return x;
    };
    double mx = 0.0;
    for (int64_t i = lane; i < n; i += 32) mx = fmax(mx, fabs(val(i)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = row_exp(mx);
    if (lane == 0) scales[j] = ldexpf(1.f, e);
    const int64_t plane = n * ldp;
    for (int64_t i = lane; i < ldp; i += 32)
        write_digits(i < n ? val(i) : 0.0, lead_bits, e, planes, slices + j * ldp + i, plane);
}

// float64 matrix -> float pair (hi = x rounded to float, lo = x - hi rounded),
// and float64 -> float; grid-stride.  The pair carries about 48 bits.
__global__ void f64_pair_kernel(const double *__restrict__ M, int64_t total, float *__restrict__ hi,
                                float *__restrict__ lo) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double x = M[t];
        const float h = (float)x;
        hi[t] = h;
        if (lo) lo[t] = (float)(x - (double)h);
    }
}

// The s = 3 A operands of the float64-storage modes from float-pair copies of a
// row-major source: X_bb(j, i) = (Mh + Ml)[j][i] s_bb(i), s_bb(i) = u(i) Ab(i, bb),
// formed in double-float float32 arithmetic (TwoProd by FMA), about 46 bits; the
// row scale bounds |hi| + |lo|, the leading digit is rint of the scaled hi part,
// and the remainder (the exact hi remainder plus the lo part, rounded once to
// float) gives the lower digits exactly as the float32 split does.  No float64
// arithmetic per entry: s_bb is formed in float64 once per block and staged as a
// float pair.  One warp per operand row; blockIdx.y indexes bb - bb0.
__global__ void __launch_bounds__(256) split_rows_g3_pair_kernel(const float *__restrict__ Mh,
                                                                 const float *__restrict__ Ml,
                                                                 const double *__restrict__ u,
                                                                 const double *__restrict__ Mb, int transAb,
                                                                 int64_t bb0, int64_t n, int64_t ldp, int lead_bits,
                                                                 int planes, __nv_bfloat16 *__restrict__ slices,
                                                                 float *__restrict__ scales) {
    extern __shared__ float2 sp[];   // [n] s_bb as (hi, lo)
    const int64_t bb = bb0 + blockIdx.y;
    slices += (int64_t)blockIdx.y * planes * n * ldp;
    scales += (int64_t)blockIdx.y * n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double v = transAb ? Mb[bb * n + i] : Mb[i * n + bb];
        if (u) v *= u[i];
        const float h = (float)v;
        sp[i] = make_float2(h, (float)(v - (double)h));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= n) return;
    const float *rh = Mh + j * n, *rl = Ml + j * n;
    auto prod = [&](int64_t i, float &vh, float &vl) {
        const float ah = rh[i], al = rl[i];
        const float2 b = sp[i];
        const float p = ah * b.x;
        const float t = fmaf(ah, b.x, -p) + fmaf(ah, b.y, al * b.x);
        vh = p + t;                 // Fast2Sum: |p| >= |t|
        vl = t - (vh - p);
    };
    float mx = 0.f;
    for (int64_t i = lane; i < n; i += 32) {
        float vh, vl;
        prod(i, vh, vl);
        mx = fmaxf(mx, fabsf(vh) + fabsf(vl));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = row_exp(mx);
    if (lane == 0) scales[j] = ldexpf(1.f, e);
    const int k = lead_bits - e;
    const int64_t plane = n * ldp;
    for (int64_t i = lane; i < ldp; i += 32) {
        float vh = 0.f, vl = 0.f;
        if (i < n) prod(i, vh, vl);
        const float yh = ldexpf(vh, k), yl = ldexpf(vl, k);   // exact scalings
        float d = rintf(yh);
        __nv_bfloat16 *dst = slices + j * ldp + i;
        dst[0] = __float2bfloat16_rn(d);                        // |d| <= 2^w: exact
        float r = (yh - d) + yl;                                // yh - d exact
        float sc = 1.f / 256.f;
        for (int p = 1; p < planes; ++p) {
            r *= 256.f;                                         // exact
            d = rintf(r);
            r -= d;                                             // exact
            dst[p * plane] = __float2bfloat16_rn(d * sc);       // exact
            sc *= (1.f / 256.f);
        }
    }
}

// Column source (X(j, i) = M[i][j] u(i)) and the tf32 copy: one block per 32
// operand rows, transposed through shared memory.
// With Mb (the s = 3 step): X(j, i) is further scaled by Ab(i, bb), bb = bb0 +
// blockIdx.y, and the digits and scales of bb go to its own region.
template <bool kSplit, typename T = float>
__global__ void __launch_bounds__(256) operand_cols_kernel(const T *__restrict__ M, int trans,
                                                           const double *__restrict__ u, int64_t n, int64_t ldp,
                                                           int lead_bits, int planes,
                                                           __nv_bfloat16 *__restrict__ slices,
                                                           float *__restrict__ scales, float *__restrict__ prep,
                                                           const T *__restrict__ Mb = nullptr, int transAb = 0,
                                                           int64_t bb0 = 0, int skip_diag = 0) {
    __shared__ T tile[32][33];
    __shared__ T rmax[8][32];
    __shared__ int rexp[32];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    const int64_t bb = bb0 + blockIdx.y;
    if (Mb) {
        slices += (int64_t)blockIdx.y * planes * n * ldp;
        scales += (int64_t)blockIdx.y * n;
    }
    auto val = [&](int64_t j, int64_t i) -> T {
        if (j >= n || i >= n || (skip_diag && i == j)) return T(0);
        T x = trans ? M[j * n + i] : M[i * n + j];
        if (u) x *= (T)u[i];
        if (Mb) x *= transAb ? Mb[bb * n + i] : Mb[i * n + bb];
        return x;
    };
    if (kSplit) {
        T mx = 0;
        if (!trans) {
            for (int64_t i = ty; i < n; i += 8) mx = fmax(mx, fabs(val(j0 + tx, i)));
            rmax[ty][tx] = mx;
        } else {
            for (int r = 0; r < 4; ++r) {
                T m2 = 0;
                for (int64_t i = tx; i < n; i += 32) m2 = fmax(m2, fabs(val(j0 + ty + 8 * r, i)));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
                if (tx == 0) tile[ty + 8 * r][0] = m2;
            }
        }
        __syncthreads();
        if (ty == 0) {
            T m = 0;
            if (!trans) {
                for (int q = 0; q < 8; ++q) m = fmax(m, rmax[q][tx]);
            } else {
                m = tile[tx][0];
            }
            const int e = row_exp(m);
            rexp[tx] = e;
            if (j0 + tx < n) scales[j0 + tx] = ldexpf(1.f, e);
        }
        __syncthreads();
    }
    const int64_t plane = n * ldp;
    for (int64_t i0 = 0; i0 < ldp; i0 += 32) {
        if (!trans) {
#pragma unroll
            for (int r = 0; r < 4; ++r) tile[tx][ty + 8 * r] = val(j0 + tx, i0 + ty + 8 * r);
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) tile[ty + 8 * r][tx] = val(j0 + ty + 8 * r, i0 + tx);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int jj = ty + 8 * r;
            const int64_t j = j0 + jj, i = i0 + tx;
            if (j >= n) continue;
            const T x = tile[jj][tx];
            if (kSplit) {
                write_digits(x, lead_bits, rexp[jj], planes, slices + j * ldp + i, plane);
            } else {
                uint32_t t;
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"((float)x));
                prep[j * ldp + i] = __uint_as_float(t);
            }
        }
        __syncthreads();
    }
}

using namespace tc;

constexpr int kBM = 128;
constexpr int kThreads = 192;

// 0 = split bf16 x3, 128 x 128 tiles, 128-byte rows, 2 stages;
// 1 = tf32; 2 = split bf16 x4, 128 x 64 tiles, 2 stages;
// 3 = split bf16 x3, 128 x 64 tiles, 3 stages;
// 4 = split bf16 x3, 128 x 128 tiles, 64-byte rows (half the k-block), 4 stages;
// 5 = split bf16 x4, 128 x 128 tiles, 64-byte rows, 3 stages;
// 6 = split bf16 x5, 128 x 128 tiles, 64-byte rows, 2 stages
// kWide (float64 storage, bf16x4 / bf16x5): one TMEM accumulator set per CTA
// instead of two, laid out [hi | mid0 | mid1 | lo]: the two slice products of
// weight 2^-8 alternate by k-block between mid0 and mid1 and the smaller ones go
// to lo.  Tensor-core float32 accumulation truncates; splitting the dominant
// correction terms over separate accumulators, each with fewer additions, cuts
// the bias that truncation leaves in a long contraction.
template <int kMode, bool kWide = false>
struct Cfg {
    static constexpr bool kTf32 = kMode == 1;
    static constexpr int kPlanes =
        (kMode == 0 || kMode == 3 || kMode == 4) ? 3 : (kMode == 1 ? 1 : (kMode == 6 ? 5 : 4));
    static constexpr int kBN = (kMode == 2 || kMode == 3) ? 64 : 128;
    static constexpr int kRowBytes = (kMode == 4 || kMode == 5 || kMode == 6) ? 64 : 128;
    static constexpr int kBKElems = kRowBytes / (kTf32 ? 4 : 2);
    static constexpr int kMmaK = kTf32 ? 8 : 16;            // 32 bytes per MMA k step
    static constexpr int kATile = kBM * kRowBytes;          // one plane of A
    static constexpr int kBTile = kBN * kRowBytes;          // one plane of B
    static constexpr int kStageBytes = kPlanes * (kATile + kBTile);
    static constexpr int kStages = kTf32 ? 6 : (kMode == 3 ? 3 : (kMode == 4 ? 4 : (kMode == 5 ? 3 : 2)));
    // accumulator sets: two (one tile's epilogue beside the next tile's MMAs)
    // wherever they fit the 512 TMEM columns
    static constexpr int kBufs = (kWide && kBN == kBM) ? 1 : 2;
    static constexpr int kAccCols = kTf32 ? kBN : (kWide ? 4 * kBN : 2 * kBN);   // hi (+ mid0, mid1) (+ lo)
    static constexpr int kTmemCols = kBufs * kAccCols;
    static constexpr int kSmem = kStages * kStageBytes + 1024 + 512;
};

// Tile t of the schedule.  Full grid: grouped raster (G tile rows per group,
// column-major inside a group, so concurrently running CTAs share A and B
// panels), in closed form.  Symmetric: the tiles tm <= tn in the same grouped
// order (a short loop over the groups).
struct TileWalk {
    int tiles_m, tiles_n, symmetric, G, batch;
    __device__ int per_product() const {
        return symmetric ? tiles_m * (tiles_m + 1) / 2 : tiles_m * tiles_n;
    }
    __device__ int count() const { return per_product() * (batch > 0 ? batch : 1); }
    // batched: product t / per_product(), then the tile within it
    __device__ void coords(int t, int &bl, int &tm, int &tn) const {
        const int per = per_product();
        bl = t / per;
        coords1(t - bl * per, tm, tn);
    }
    __device__ void coords1(int t, int &tm, int &tn) const {
        if (symmetric) {
            // the tiles on or above the diagonal in groups of G tile rows; inside a
            // group column by column, each column's rows of the group (a triangle over
            // the group's first G columns, then full columns), so that the CTAs of a
            // wave share G A panels and a few B panels, as in the full-grid raster
            const int T = tiles_m;
            int r0 = 0;
            for (;;) {
                const int g = min(G, T - r0);
                const int tri = g * (g + 1) / 2;
                const int cnt = tri + g * (T - r0 - g);
                if (t < cnt || r0 + g >= T) {
                    if (t < tri) {
                        int c = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
                        while (c > 0 && c * (c + 1) / 2 > t) --c;
                        while ((c + 1) * (c + 2) / 2 <= t) ++c;
                        tm = r0 + (t - c * (c + 1) / 2);
                        tn = r0 + c;
                    } else {
                        const int v = t - tri;
                        tm = r0 + v % g;
                        tn = r0 + g + v / g;
                    }
                    return;
                }
                t -= cnt;
                r0 += g;
            }
        }
        const int per_group = G * tiles_n;
        const int group = t / per_group;
        const int first = group * G;
        const int gm = min(G, tiles_m - first);
        const int rr = t - group * per_group;
        tm = first + rr % gm;
        tn = rr / gm;
    }
};

// The group entry holding tile t: start[p] <= t < start[p + 1] (binary search).
__device__ __forceinline__ int group_find(const int *start, int count, int t) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// kGroup: one persistent launch over the tiles of many products (g.gcount group
// entries, each with its own sizes, operands, tensor maps and reductions in
// global memory); otherwise one product (or one s = 3 batch) from g itself.
template <int kMode, bool kWide = false, bool kGroup = false>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapB2, TcGemmArgs g) {
    using C = Cfg<kMode, kWide>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t bar_base = base + C::kStages * C::kStageBytes;
    auto full_bar = [&](int s) { return bar_base + 8u * s; };
    auto empty_bar = [&](int s) { return bar_base + 8u * (C::kStages + s); };
    auto tfull_bar = [&](int b) { return bar_base + 8u * (2 * C::kStages + b); };
    auto tempty_bar = [&](int b) { return bar_base + 8u * (2 * C::kStages + 2 + b); };
    const uint32_t abort_bar = bar_base + 8u * (2 * C::kStages + 4);   // MMAs in flight at an abort
    uint8_t *misc = gbase + C::kStages * C::kStageBytes + 8 * (2 * C::kStages + 5);
    volatile uint32_t *tmem_holder = (volatile uint32_t *)misc;
    volatile int *abort_flag = (volatile int *)(misc + 4);
    volatile uint32_t *issued_cnt = (volatile uint32_t *)(misc + 8);
    volatile uint32_t *consumed_cnt = (volatile uint32_t *)(misc + 12);
    double *wred = (double *)(misc + 16);   // [4 warps][4 reductions]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = g.n;
    // the window of the product this launch computes (the whole product by default)
    const bool win = g.rows > 0;
    const int64_t row0 = win ? g.row0 : 0, col0 = win ? g.col0 : 0;
    const int64_t jend = win ? row0 + g.rows : n, kend = win ? col0 + g.cols : n;
    const int num_k = (int)(g.ldp / C::kBKElems);
    const long long wlim = g.wait_limit > 0 ? g.wait_limit : kWaitLimit;
    TileWalk walk{(int)((jend - row0 + kBM - 1) / kBM), (int)((kend - col0 + C::kBN - 1) / C::kBN), g.symmetric,
                  g.group_rows > 0 ? g.group_rows : 8, g.batch};
    // work units: the tiles, except that the last g.split_tail tiles of the schedule
    // are split into two halves of kBN / 2 columns, so that the last wave of the
    // persistent grid is (nearly) full
    // a row shard (g.tile_hi > 0) takes the tiles tile_lo .. tile_hi - 1 of the walk
    const int t_lo = g.tile_hi > 0 ? g.tile_lo : 0;
    const int n_tiles = g.tile_hi > 0 ? g.tile_hi - g.tile_lo : walk.count();
    const int split_tail = g.split_tail;
    const int total_tiles = kGroup ? g.gstart[g.gcount] : n_tiles + split_tail;
    constexpr int kHalf = C::kBN / 2;
    // group entry p of tile t and the tile's coordinates in that product's walk
    auto gunit = [&](int t, int &p, int &tm, int &tn) {
        p = group_find(g.gstart, g.gcount, t);
        const TcGemmArgs &a = g.gargs[p];
        const TileWalk w{(int)((a.n + kBM - 1) / kBM), (int)((a.n + C::kBN - 1) / C::kBN), a.symmetric,
                         a.group_rows > 0 ? a.group_rows : 8, 0};
        int bl;
        w.coords(t - g.gstart[p], bl, tm, tn);
    };
    auto unit = [&](int t, int &bl, int &tm, int &tn, int &c_off, int &width) {
        const int f = n_tiles - split_tail;
        if (t < f) {
            walk.coords(t_lo + t, bl, tm, tn);
            c_off = 0;
            width = C::kBN;
        } else {
            const int v = t - f;
            walk.coords(t_lo + f + (v >> 1), bl, tm, tn);
            c_off = (v & 1) * kHalf;
            width = kHalf;
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), 4);
        }
        mbar_init(abort_bar, 1);
        *abort_flag = 0;
        *issued_cnt = 0;
        *consumed_cnt = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void *)tmem_holder)),
                     "r"(C::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            uint32_t it = 0;
            // g.debug_stall (a test hook, off by default): issue no copy at all, so
            // that the MMA warp's first wait runs out with nothing in flight
            for (int t = g.debug_stall ? total_tiles : (int)blockIdx.x; t < total_tiles && !*abort_flag;
                 t += gridDim.x) {
                int bl = 0, tm, tn, c_off = 0, width = C::kBN, nk = num_k;
                const CUtensorMap *mA = &mapA, *mB = &mapB, *mB2 = &mapB2;
                if constexpr (kGroup) {
                    int p;
                    gunit(t, p, tm, tn);
                    nk = (int)(g.gargs[p].ldp / C::kBKElems);
                    mA = reinterpret_cast<const CUtensorMap *>(g.gmaps) + 2 * p;
                    mB = mA + 1;
                } else {
                    unit(t, bl, tm, tn, c_off, width);
                }
                const int za = bl * C::kPlanes;   // the product's A planes (batched s = 3 step)
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = it % C::kStages;
                    if (it >= (uint32_t)C::kStages &&
                        !mbar_wait(empty_bar(s), ((it / C::kStages) - 1) & 1, abort_flag, wlim))
                        break;
                    const uint32_t sa = base + s * C::kStageBytes;
                    const uint32_t sb = sa + C::kPlanes * C::kATile;
                    mbar_expect_tx(full_bar(s), width == C::kBN ? C::kStageBytes
                                                                : C::kPlanes * (C::kATile + C::kBTile / 2));
                    tma_load_3d(sa, mA, kb * C::kBKElems, tm * kBM, za, full_bar(s));
                    if (width == C::kBN) tma_load_3d(sb, mB, kb * C::kBKElems, tn * C::kBN, 0, full_bar(s));
                    else tma_load_3d(sb, mB2, kb * C::kBKElems, tn * C::kBN + c_off, 0, full_bar(s));
                    *issued_cnt = it + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            constexpr uint32_t idesc_full = make_idesc(C::kTf32 ? 2u : 1u, kBM, C::kBN);
            constexpr uint32_t idesc_half = make_idesc(C::kTf32 ? 2u : 1u, kBM, kHalf);
            uint32_t it = 0, tcount = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
                int bl = 0, tm, tn, c_off = 0, width = C::kBN, nk = num_k;
                if constexpr (kGroup) {
                    int p;
                    gunit(t, p, tm, tn);
                    nk = (int)(g.gargs[p].ldp / C::kBKElems);
                } else {
                    unit(t, bl, tm, tn, c_off, width);
                }
                (void)bl;
                const uint32_t idesc = width == C::kBN ? idesc_full : idesc_half;
                const uint32_t b_plane = width == C::kBN ? C::kBTile : C::kBTile / 2;   // bytes per B plane
                const int buf = tcount % C::kBufs;
                if (tcount >= (uint32_t)C::kBufs &&
                    !mbar_wait(tempty_bar(buf), ((tcount / C::kBufs) - 1) & 1, abort_flag, wlim)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_hi = tmem + buf * C::kAccCols;
                const uint32_t d_lo = d_hi + (kWide ? 3 : 1) * C::kBN;
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = it % C::kStages;
                    if (!mbar_wait(full_bar(s), (it / C::kStages) & 1, abort_flag, wlim)) {
                        ok = false;
                        break;
                    }
                    *consumed_cnt = it + 1;
                    tc_fence_after();
                    const uint32_t sa = base + s * C::kStageBytes;
                    const uint32_t sb = sa + C::kPlanes * C::kATile;
#pragma unroll
                    for (int kk = 0; kk < C::kBKElems / C::kMmaK; ++kk) {
                        const uint32_t koff = kk * 32;
                        const uint32_t acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
                        if constexpr (C::kTf32) {
                            mma<true>(d_hi, desc_sw<C::kRowBytes>(sa + koff), desc_sw<C::kRowBytes>(sb + koff), idesc, acc0);
                        } else {
                            uint64_t ad[C::kPlanes], bd[C::kPlanes];
#pragma unroll
                            for (int p = 0; p < C::kPlanes; ++p) {
                                ad[p] = desc_sw<C::kRowBytes>(sa + p * C::kATile + koff);
                                bd[p] = desc_sw<C::kRowBytes>(sb + p * b_plane + koff);
                            }
                            // leading product into its own accumulator; every slice
                            // pair of weight 2^-8 .. 2^-8 (S - 1) into the other
                            mma<false>(d_hi, ad[0], bd[0], idesc, acc0);
                            if constexpr (kWide) {
                                const uint32_t d_mid = d_hi + (1 + (kb & 1)) * C::kBN;
                                const uint32_t accm = (kb > 1 || kk > 0) ? 1u : 0u;
                                mma<false>(d_mid, ad[0], bd[1], idesc, accm);
                                mma<false>(d_mid, ad[1], bd[0], idesc, 1u);
                                if (C::kPlanes > 2) mma<false>(d_lo, ad[0], bd[2], idesc, acc0);
                            } else {
                                mma<false>(d_lo, ad[0], bd[1], idesc, acc0);
                                mma<false>(d_lo, ad[1], bd[0], idesc, 1u);
                            }
#pragma unroll
                            for (int sum = 2; sum < C::kPlanes; ++sum) {
#pragma unroll
                                for (int i = 0; i <= sum; ++i) {
                                    if (kWide && sum == 2 && i == 0) continue;   // issued above
                                    mma<false>(d_lo, ad[i], bd[sum - i], idesc, 1u);
                                }
                            }
                        }
                    }
                    mma_commit(empty_bar(s));   // frees the stage when these MMAs complete
                }
                if (!ok) break;
                mma_commit(tfull_bar(buf));     // accumulator buffer ready for the epilogue
                ++tcount;
            }
        }
    } else {
        // ---------------- epilogue warps 2..5: TMEM lanes 32 (warp % 4) ..
        const int q = warp & 3;
        const int row = 32 * q + lane;
        double total[4] = {0.0, 0.0, 0.0, 0.0};
        uint32_t tcount = 0;
        // one tile's epilogue; g and the sizes are the product's (a group entry's in
        // a grouped launch)
        auto epi_tile = [&](const TcGemmArgs &g, const int64_t n, const int64_t jend, const int64_t kend,
                            const int num_k, const int64_t row0, const int64_t col0, int bl, int tm, int tn,
                            int c_off, int width) -> bool {
            const int64_t bb = g.bb0 + bl;   // batched s = 3 step: this product's index
            const float *Wbd = (const float *)g.Wbd;
            const int tWbd = g.transWbd;
            const int buf = tcount % C::kBufs;
            // one lane polls (with back-off: the main loop of a tile takes tens of
            // microseconds) so the waiting warps leave the issue slots to the TMA
            // and MMA warps
            int waited = 0;
            if (lane == 0) waited = mbar_wait(tfull_bar(buf), (tcount / C::kBufs) & 1, abort_flag, wlim) ? 1 : 0;
            waited = __shfl_sync(0xffffffffu, waited, 0);
            if (!waited || *abort_flag) return false;
            tc_fence_after();
            const int64_t j = row0 + (int64_t)tm * kBM + row;
            const bool jok = j < jend;
            const float rs = jok ? (C::kTf32 ? 1.f : ldexpf(g.scaleA[(int64_t)bl * n + j], -2 * g.lead_bits)) : 0.f;
            // the row's scale 2^row_e (with the leading digits' weight): scaleA holds
            // powers of two (0 for a zero row, whose entries are then 0)
            const float sa = jok && !C::kTf32 ? g.scaleA[(int64_t)bl * n + j] : 0.f;
            const int row_e = sa != 0.f ? ilogbf(sa) - 2 * g.lead_bits : 0;
            const uint32_t taddr = tmem + buf * C::kAccCols + ((uint32_t)(32 * q) << 16);
            double tile_acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 1
            for (int c0 = 0; c0 < width; c0 += 16) {
                uint32_t hi[16], lo[16], m0[16], m1[16];
                tmem_ld16(taddr + c0, hi);
                if constexpr (kWide) {
                    tmem_ld16(taddr + C::kBN + c0, m0);
                    tmem_ld16(taddr + 2 * C::kBN + c0, m1);
                    tmem_ld16(taddr + 3 * C::kBN + c0, lo);
                } else {
                    if (!C::kTf32) tmem_ld16(taddr + C::kBN + c0, lo);
                }
                tmem_wait_ld();
                const int64_t k0 = col0 + (int64_t)tn * C::kBN + c_off + c0;
                if (kWide && !g.wide_f32) {
                    // float64 storage.  The four accumulators are summed exactly in
                    // float32 pairs (TwoSum; mid1 holds the odd k-blocks' products,
                    // nothing when there is one), and each half becomes a float64
                    // scaled by the power-of-two row and column scales through its
                    // bit fields: one float64 addition per entry, where converting and
                    // adding the accumulators in float64 took nine operations of this
                    // part's slow float64 pipe
                    double v[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const int64_t k = k0 + c;
                        float s, t, t2;
                        two_sum(__uint_as_float(hi[c]), __uint_as_float(m0[c]), s, t);
                        if (num_k > 1) {
                            two_sum(s, __uint_as_float(m1[c]), s, t2);
                            t = __fadd_rn(t, t2);
                        }
                        if (C::kPlanes > 2) {
                            two_sum(s, __uint_as_float(lo[c]), s, t2);
                            t = __fadd_rn(t, t2);
                        }
                        const float sb = k < kend ? g.scaleB[k] : 0.f;
                        if (sb == 0.f || sa == 0.f) {
                            v[c] = 0.0;
                        } else {
                            const int e = ilogbf(sb) + row_e;
                            v[c] = f2d_scaled(s, e) + f2d_scaled(t, e);
                        }
                    }
                    if ((g.dA || g.dB) && jok) {
                        // the terms i = j and i = k of operands split without their
                        // diagonal, each one fused multiply-add
                        const double *MA = (const double *)g.MA, *MB = (const double *)g.MB;
                        const double dAj = g.dA ? g.dA[j] : 0.0;
                        const double aj = dAj * (g.uB ? g.uB[j] : 1.0);
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const int64_t k = k0 + c;
                            if (k >= kend) continue;
                            double w = v[c];
                            const double dBk = g.dB ? g.dB[k] : 0.0;
                            if (aj != 0.0) w = fma(aj, g.rowB ? MB[j * n + k] : MB[k * n + j], w);
                            if (dBk != 0.0)
                                w = fma(g.rowA ? MA[j * n + k] : MA[k * n + j], g.uA ? g.uA[k] * dBk : dBk, w);
                            if (k == j) w -= dAj * dBk;
                            v[c] = w;
                        }
                    }
                    if (g.C && jok) {
                        double *Cd = (double *)g.C;
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            if (k0 + c < kend) Cd[j * n + k0 + c] = v[c];
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        if (r >= g.nred) break;
                        const double *W = (const double *)g.red[r].W;
                        const double *bv = g.red[r].b;
                        const double *Wbd = (const double *)g.Wbd;
                        const int tW = g.red[r].transW, pw = g.red[r].pow;
                        double part = 0.0;
                        if (jok) {
#pragma unroll
                            for (int c = 0; c < 16; ++c) {
                                const int64_t k = k0 + c;
                                if (k >= kend) continue;
                                double w = bv ? bv[k] : 1.0;
                                if (W) w *= tW ? W[k * n + j] : W[j * n + k];
                                if (Wbd) w *= g.transWbd ? Wbd[k * n + bb] : Wbd[bb * n + k];
                                const double x = pw == 2 ? v[c] * v[c] : v[c];
                                part = fma(x, w, part);
                            }
                        }
                        tile_acc[r] += part;
                    }
                } else {
                    // float32 epilogue: the float32-storage modes, and the s = 3 step of
                    // the float64-storage modes (float32 copies of the weights; the
                    // accumulators summed smallest first, rounded once per entry)
                    float v[16];
    #pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        float x = __uint_as_float(hi[c]);
                        if (!C::kTf32) {
                            const int64_t k = k0 + c;
                            float corr = __uint_as_float(lo[c]);
                            if constexpr (kWide)
                                corr = (num_k > 1 ? __uint_as_float(m1[c]) : 0.f) +
                                       ((C::kPlanes > 2 ? corr : 0.f) + __uint_as_float(m0[c]));
                            x = (x + corr) * (k < kend ? g.scaleB[k] : 0.f);
                        }
                        v[c] = x * rs;
                    }
                    if ((g.dA || g.dB) && jok) {
                        // the terms i = j and i = k of operands split without their diagonal
                        const float *MA = (const float *)g.MA, *MB = (const float *)g.MB;
                        const float dAj = g.dA ? (float)g.dA[j] : 0.f;
                        float dBk[16];
                        bool anyB = false;
    #pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            dBk[c] = (g.dB && k0 + c < kend) ? (float)g.dB[k0 + c] : 0.f;
                            anyB |= dBk[c] != 0.f;
                        }
                        // rows j of the sources, 16-byte loads where they lie inside
                        const bool full = (k0 + 16 <= kend) && ((n & 3) == 0);
                        auto row16 = [&](const float *M, int rowf, float (&r)[16]) {
                            if (rowf && full) {
                                const float4 *p4 = reinterpret_cast<const float4 *>(M + j * n + k0);
    #pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    const float4 t4 = p4[q];
                                    r[4 * q] = t4.x, r[4 * q + 1] = t4.y, r[4 * q + 2] = t4.z, r[4 * q + 3] = t4.w;
                                }
                            } else {
    #pragma unroll
                                for (int c = 0; c < 16; ++c)
                                    r[c] = k0 + c < kend ? (rowf ? M[j * n + k0 + c] : M[(k0 + c) * n + j]) : 0.f;
                            }
                        };
                        float xb[16], xa[16];
                        if (dAj != 0.f) {
                            row16(MB, g.rowB, xb);
                            const float ub = g.uB ? (float)g.uB[j] : 1.f;
    #pragma unroll
                            for (int c = 0; c < 16; ++c) v[c] += dAj * xb[c] * ub;
                        }
                        if (anyB) {
                            if (dAj != 0.f && MA == MB && g.rowA == g.rowB) {
    #pragma unroll
                                for (int c = 0; c < 16; ++c) xa[c] = xb[c];
                            } else {
                                row16(MA, g.rowA, xa);
                            }
    #pragma unroll
                            for (int c = 0; c < 16; ++c)
                                v[c] += xa[c] * (g.uA && k0 + c < kend ? (float)g.uA[k0 + c] : 1.f) * dBk[c];
                        }
    #pragma unroll
                        for (int c = 0; c < 16; ++c)
                            if (k0 + c == j) v[c] -= dAj * dBk[c];
                    }
                    if (g.C && jok) {
    #pragma unroll
                        for (int c = 0; c < 16; ++c)
                            if (k0 + c < kend) ((float *)g.C)[j * n + k0 + c] = v[c];
                    }
                    // the 16 columns lie inside the matrix and rows are 16-byte aligned:
                    // weights are read as float4
                    const bool full = (k0 + 16 <= kend) && ((n & 3) == 0);
    #pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        if (r >= g.nred) break;
                        const float *W = (const float *)g.red[r].W;
                        const double *bv = g.red[r].b;
                        const int tW = g.red[r].transW, pw = g.red[r].pow;
                        float part = 0.f;
                        if (jok) {
                            float w[16];
                            if (W && !tW && full) {
                                const float4 *p4 = reinterpret_cast<const float4 *>(W + j * n + k0);
    #pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    const float4 t4 = p4[q];
                                    w[4 * q] = t4.x, w[4 * q + 1] = t4.y, w[4 * q + 2] = t4.z, w[4 * q + 3] = t4.w;
                                }
                            } else {
    #pragma unroll
                                for (int c = 0; c < 16; ++c) {
                                    const int64_t k = k0 + c;
                                    w[c] = k < kend ? (W ? (tW ? W[k * n + j] : W[j * n + k]) : 1.f) : 0.f;
                                }
                            }
                            if (bv) {
    #pragma unroll
                                for (int c = 0; c < 16; ++c) w[c] *= k0 + c < kend ? (float)bv[k0 + c] : 0.f;
                            }
                            if (Wbd) {
                                if (!tWbd && full) {
                                    const float4 *p4 = reinterpret_cast<const float4 *>(Wbd + bb * n + k0);
    #pragma unroll
                                    for (int q = 0; q < 4; ++q) {
                                        const float4 t4 = p4[q];
                                        w[4 * q] *= t4.x, w[4 * q + 1] *= t4.y, w[4 * q + 2] *= t4.z, w[4 * q + 3] *= t4.w;
                                    }
                                } else {
    #pragma unroll
                                    for (int c = 0; c < 16; ++c) {
                                        const int64_t k = k0 + c;
                                        if (k < kend) w[c] *= tWbd ? Wbd[k * n + bb] : Wbd[bb * n + k];
                                    }
                                }
                            }
    #pragma unroll
                            for (int c = 0; c < 16; ++c) {
                                const float x = pw == 2 ? v[c] * v[c] : v[c];
                                part = fmaf(x, w[c], part);
                            }
                        }
                        tile_acc[r] += (double)part;
                    }
                }
                }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(buf));
            double wgt = ((g.symmetric && tm != tn) ? 2.0 : 1.0) * (g.wscale != 0.0 ? g.wscale : 1.0);
            if (g.ub) wgt *= g.ub[bb];
            double wbc = 1.0;
            if (g.Wbc && jok) {
                const int64_t wi = g.transWbc ? j * n + bb : bb * n + j;
                wbc = (kWide && !g.wide_f32) ? ((const double *)g.Wbc)[wi] : (double)((const float *)g.Wbc)[wi];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r >= g.nred) break;
                const double aj = (g.red[r].a && jok) ? g.red[r].a[j] : 1.0;
                const double x = tile_acc[r] * aj * wbc * wgt;
                if constexpr (kGroup) {
                    // a group entry's own output: this warp's share of the tile
                    const double sw = warp_sum(x);
                    if (lane == 0 && !*abort_flag) atomicAdd(g.red[r].out, sw);
                } else {
                    total[r] += x;
                }
            }
            return true;
        };
        for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
            bool ok;
            if constexpr (kGroup) {
                int p, tm, tn;
                gunit(t, p, tm, tn);
                const TcGemmArgs &a = g.gargs[p];
                ok = epi_tile(a, a.n, a.n, a.n, (int)(a.ldp / C::kBKElems), 0, 0, 0, tm, tn, 0, C::kBN);
            } else {
                int bl, tm, tn, c_off, width;
                unit(t, bl, tm, tn, c_off, width);
                ok = epi_tile(g, n, jend, kend, num_k, row0, col0, bl, tm, tn, c_off, width);
            }
            if (!ok) break;
            ++tcount;
        }
        // reduce the four epilogue warps' partial sums
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const double s = warp_sum(total[r]);
            if (lane == 0) wred[(warp - 2) * 4 + r] = s;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (warp == 2 && lane < g.nred && !*abort_flag) {
            const double s = wred[lane] + wred[4 + lane] + wred[8 + lane] + wred[12 + lane];
            atomicAdd(g.red[lane].out, s);
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (*abort_flag) {
        if (warp == 1 && lane == 0) {
            // MMAs issued before the abort may still read shared memory and write
            // TMEM: one more commit by their issuing thread arrives on abort_bar
            // once all of them are done; the TMEM is freed only after that
            mma_commit(abort_bar);
            mbar_drain(abort_bar, 0, wlim);
        }
        if (threadIdx.x == 0) {
            if (g.err) atomicOr(g.err, kErrWordTimeout);
            if constexpr (kGroup)
                for (int p = 0; p < g.gcount; ++p)
                    if (g.gargs[p].err) atomicOr(g.gargs[p].err, kErrWordTimeout);
            // wait (bounded in time) for the copies issued but never consumed, before
            // the shared memory they land in is released
            for (uint32_t i = *consumed_cnt; i < *issued_cnt; ++i)
                if (!mbar_drain(full_bar(i % C::kStages), (i / C::kStages) & 1, wlim)) break;
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kTmemCols));
    }
}

// ------------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

}  // namespace

bool make_map_planes(CUtensorMap *map, const void *ptr, bool bf16, int planes, int total_planes, int64_t rows,
                     int64_t ldp, int box_rows, int row_bytes) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return false;
    const int esz = bf16 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)ldp, (cuuint64_t)rows, (cuuint64_t)total_planes};
    cuuint64_t strides[2] = {(cuuint64_t)(ldp * esz), (cuuint64_t)(rows * ldp * esz)};
    cuuint32_t box[3] = {(cuuint32_t)(row_bytes / esz), (cuuint32_t)box_rows, (cuuint32_t)planes};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                     const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int sm_count() {
    static int cnt[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (!cnt[dev]) {
        int c = 0;
        if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = 148;
        cnt[dev] = c;
    }
    return cnt[dev];
}

namespace {

long long g_debug_wait_limit = 0;
int g_debug_stall = 0;

template <int kMode, bool kWide = false>
cudaError_t launch_tc(const TcGemmArgs &g0, cudaStream_t s) {
    using C = Cfg<kMode, kWide>;
    TcGemmArgs g = g0;
    g.wait_limit = g_debug_wait_limit;
    g.debug_stall = g_debug_stall;
    if (C::kBN != kBM || g.C) g.symmetric = 0;
    if (g.nred < 0 || g.nred > 4) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    const bool bf16 = !C::kTf32;
    if (g.batch > 0 && (g.C || g.nred != 1)) return cudaErrorInvalidValue;
    if (g.wide_f32 && (!kWide || g.C)) return cudaErrorInvalidValue;
    if ((g.dA || g.dB) && (g.batch > 0 || (g.dA && !g.MB) || (g.dB && !g.MA))) return cudaErrorInvalidValue;
    const int za = g.batch > 0 ? g.batch : 1;
    CUtensorMap mb2;
    // a window: rows row0 .. row0 + rows - 1 and columns col0 .. col0 + cols - 1 of
    // the product, reductions only; its operands hold just those rows
    const bool win = g.rows > 0;
    if (win && (g.cols < 1 || g.row0 < 0 || g.col0 < 0 || g.row0 + g.rows > g.n || g.col0 + g.cols > g.n ||
                g.C || g.batch > 0 || g.dA || g.dB || g.shard_count > 1 ||
                (g.symmetric && (g.row0 != g.col0 || g.rows != g.cols))))
        return cudaErrorInvalidValue;
    const int64_t ra = win ? g.rows : g.n, rb = win ? g.cols : g.n;
    if (!make_map_planes(&ma, g.opA, bf16, C::kPlanes, za * C::kPlanes, ra, g.ldp, kBM, C::kRowBytes) ||
        !make_map_planes(&mb, g.opB, bf16, C::kPlanes, C::kPlanes, rb, g.ldp, C::kBN, C::kRowBytes) ||
        !make_map_planes(&mb2, g.opB, bf16, C::kPlanes, C::kPlanes, rb, g.ldp, C::kBN / 2, C::kRowBytes))
        return cudaErrorInvalidValue;
    static std::atomic<bool> attr[64];   // per device, set once; atomic: host threads may launch concurrently
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<kMode, kWide>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             C::kSmem);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    const int64_t tm = (ra + kBM - 1) / kBM, tn = (rb + C::kBN - 1) / C::kBN;
    int64_t tiles = (g.symmetric ? tm * (tm + 1) / 2 : tm * tn) * za;
    g.tile_lo = g.tile_hi = 0;
    if (g.shard_count > 1) {
        if (g.C || g.shard_rank < 0 || g.shard_rank >= g.shard_count) return cudaErrorInvalidValue;
        const int64_t lo = tiles * g.shard_rank / g.shard_count, hi = tiles * (g.shard_rank + 1) / g.shard_count;
        if (hi <= lo) return cudaSuccess;   // nothing in this range
        g.tile_lo = (int)lo;
        g.tile_hi = (int)hi;
        tiles = hi - lo;
    }
    // half tiles for the last, partly filled wave: with R tiles left over after the
    // full waves, split R of them when 2R still fits one wave (all of them, up to
    // the SM count, when there is less than one wave)
    const int64_t S = sm_count();
    int64_t split = 0;
    if (tiles <= S) split = std::min(tiles, S - tiles);
    else if (tiles % S != 0 && 2 * (tiles % S) <= S) split = tiles % S;
    g.split_tail = (int)split;
    const int64_t units = tiles + split;
    const int grid = (int)(units < S ? units : S);
    tc_gemm_kernel<kMode, kWide><<<grid, kThreads, C::kSmem, s>>>(ma, mb, mb2, g);
    return cudaGetLastError();
}

}  // namespace

void set_tc_debug(long long wait_limit, int stall) {
    g_debug_wait_limit = wait_limit > 0 ? wait_limit : 0;
    g_debug_stall = stall != 0;
}

long long tc_debug_wait_limit() { return g_debug_wait_limit; }

cudaError_t launch_split(const void *M, bool wide, int trans, const double *u, int64_t n, int64_t ldp,
                         int lead_bits, int planes, void *slices, float *scales, double *diag_out, cudaStream_t s) {
    const int sd = diag_out ? 1 : 0;
    if (trans) {
        if (wide)
            split_rows_kernel<double><<<(unsigned)((n + 7) / 8), 256, 0, s>>>(
                (const double *)M, u, n, ldp, lead_bits, planes, (__nv_bfloat16 *)slices, scales, diag_out);
        else
            split_rows_kernel<float><<<(unsigned)((n + 7) / 8), 256, 0, s>>>(
                (const float *)M, u, n, ldp, lead_bits, planes, (__nv_bfloat16 *)slices, scales, diag_out);
        return cudaGetLastError();
    } else {
        dim3 grid((unsigned)((n + 31) / 32)), block(32, 8);
        if (wide)
            operand_cols_kernel<true, double><<<grid, block, 0, s>>>((const double *)M, 0, u, n, ldp, lead_bits,
                                                                     planes, (__nv_bfloat16 *)slices, scales, nullptr,
                                                                     nullptr, 0, 0, sd);
        else
            operand_cols_kernel<true, float><<<grid, block, 0, s>>>((const float *)M, 0, u, n, ldp, lead_bits, planes,
                                                                    (__nv_bfloat16 *)slices, scales, nullptr, nullptr,
                                                                    0, 0, sd);
    }
    if (diag_out) {
        const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
        if (wide) operand_diag_kernel<double><<<blocks, 256, 0, s>>>((const double *)M, u, n, diag_out);
        else operand_diag_kernel<float><<<blocks, 256, 0, s>>>((const float *)M, u, n, diag_out);
    }
    return cudaGetLastError();
}

cudaError_t launch_split_g3(const void *Mv, bool wide, int trans, const double *u, const void *Mbv, int transAb,
                            int64_t bb0, int nb, int64_t n, int64_t ldp, int lead_bits, int planes, void *slices,
                            float *scales, cudaStream_t s) {
    if (nb < 1 || nb > 65535) return cudaErrorInvalidValue;
    {
        // The split of the next batch runs beside the persistent GEMM, which holds
        // most of each SM's shared memory: these kernels ask for the same L1 /
        // shared-memory split, so that their CTAs can share an SM with the GEMM's.
        static std::atomic<bool> carve[64];   // per device, set once; atomic: host threads may launch concurrently
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!carve[dev]) {
            const void *fns[] = {(const void *)split_rows_g3_kernel, (const void *)split_rows_g3_wide_kernel,
                                 (const void *)operand_cols_kernel<true, double>,
                                 (const void *)operand_cols_kernel<true, float>};
            for (const void *f : fns) {
                cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                     (int)cudaSharedmemCarveoutMaxShared);
                if (e != cudaSuccess) return e;
            }
            carve[dev] = true;
        }
    }
    if (wide) {
        if (trans) {
            dim3 grid((unsigned)((n + 7) / 8), (unsigned)nb);
            split_rows_g3_wide_kernel<<<grid, 256, 0, s>>>((const double *)Mv, u, (const double *)Mbv, transAb, bb0, n,
                                                          ldp, lead_bits, planes, (__nv_bfloat16 *)slices, scales);
        } else {
            dim3 grid((unsigned)((n + 31) / 32), (unsigned)nb), block(32, 8);
            operand_cols_kernel<true, double><<<grid, block, 0, s>>>((const double *)Mv, trans, u, n, ldp, lead_bits,
                                                                     planes, (__nv_bfloat16 *)slices, scales, nullptr,
                                                                     (const double *)Mbv, transAb, bb0);
        }
        return cudaGetLastError();
    }
    const float *M = (const float *)Mv, *Mb = (const float *)Mbv;
    if (trans && n <= 32768) {
        // A(i, j) = M[j][i]: operand rows are source rows
        const int smem = (int)(sizeof(float) * n);
        if (smem > 48 * 1024) {
            static std::atomic<bool> attr[64];   // per device, set once; atomic: host threads may launch concurrently
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
            if (!attr[dev]) {
                cudaError_t e = cudaFuncSetAttribute(split_rows_g3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     32768 * (int)sizeof(float));
                if (e != cudaSuccess) return e;
                attr[dev] = true;
            }
        }
        dim3 grid((unsigned)((n + 7) / 8), (unsigned)nb);
        split_rows_g3_kernel<<<grid, 256, smem, s>>>(M, u, Mb, transAb, bb0, n, ldp, lead_bits, planes,
                                                    (__nv_bfloat16 *)slices, scales);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)nb), block(32, 8);
    operand_cols_kernel<true, float><<<grid, block, 0, s>>>(M, trans, u, n, ldp, lead_bits, planes,
                                                     (__nv_bfloat16 *)slices, scales, nullptr, Mb, transAb, bb0);
    return cudaGetLastError();
}

cudaError_t launch_f64_pair(const double *M, int64_t total, float *hi, float *lo, cudaStream_t s) {
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 8 * (int64_t)sm_count());
    f64_pair_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(M, total, hi, lo);
    return cudaGetLastError();
}

cudaError_t launch_split_g3_pair(const float *Mh, const float *Ml, const double *u, const double *Mb, int transAb,
                                 int64_t bb0, int nb, int64_t n, int64_t ldp, int lead_bits, int planes, void *slices,
                                 float *scales, cudaStream_t s) {
    if (nb < 1 || nb > 65535 || n > kPairSplitMaxN) return cudaErrorInvalidValue;
    static std::atomic<bool> attr[64];   // per device, set once; atomic: host threads may launch concurrently
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(split_rows_g3_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(float2) * kPairSplitMaxN));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(split_rows_g3_pair_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    dim3 grid((unsigned)((n + 7) / 8), (unsigned)nb);
    split_rows_g3_pair_kernel<<<grid, 256, sizeof(float2) * n, s>>>(Mh, Ml, u, Mb, transAb, bb0, n, ldp, lead_bits,
                                                                    planes, (__nv_bfloat16 *)slices, scales);
    return cudaGetLastError();
}

cudaError_t launch_prep(const float *M, int trans, const double *u, int64_t n, int64_t ldp, float *out,
                        cudaStream_t s) {
    dim3 grid((unsigned)((n + 31) / 32)), block(32, 8);
    operand_cols_kernel<false, float><<<grid, block, 0, s>>>(M, trans, u, n, ldp, 0, 1, nullptr, nullptr, out);
    return cudaGetLastError();
}

namespace {

size_t round_to(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The device image of a group: per entry the A and B tensor maps (128 bytes each,
// 64-byte aligned), then the entries' arguments, then the tile prefix sums.
size_t group_maps_bytes(int count) { return round_to((size_t)count * 2 * sizeof(CUtensorMap), 256); }
size_t group_args_bytes(int count) { return round_to((size_t)count * sizeof(TcGemmArgs), 256); }

template <int kMode>
int group_image_t(const TcGemmArgs *items, int count, const void *dev_base, std::vector<char> &host) {
    using C = Cfg<kMode, false>;
    host.assign(gemm_group_bytes(count), 0);
    CUtensorMap *maps = reinterpret_cast<CUtensorMap *>(host.data());
    TcGemmArgs *args = reinterpret_cast<TcGemmArgs *>(host.data() + group_maps_bytes(count));
    int *start = reinterpret_cast<int *>(host.data() + group_maps_bytes(count) + group_args_bytes(count));
    int64_t total = 0;
    start[0] = 0;
    for (int p = 0; p < count; ++p) {
        TcGemmArgs a = items[p];
        if (a.batch > 0 || a.rows > 0 || a.shard_count > 1 || a.wide || a.wide_f32 || a.nred < 0 || a.nred > 4)
            return -1;
        if (C::kBN != kBM || a.C) a.symmetric = 0;
        if (!make_map_planes(&maps[2 * p], a.opA, true, C::kPlanes, C::kPlanes, a.n, a.ldp, kBM, C::kRowBytes) ||
            !make_map_planes(&maps[2 * p + 1], a.opB, true, C::kPlanes, C::kPlanes, a.n, a.ldp, C::kBN,
                             C::kRowBytes))
            return -1;
        const int64_t tm = (a.n + kBM - 1) / kBM, tn = (a.n + C::kBN - 1) / C::kBN;
        total += a.symmetric ? tm * (tm + 1) / 2 : tm * tn;
        if (total > (int64_t)1 << 30) return -1;
        start[p + 1] = (int)total;
        args[p] = a;
    }
    (void)dev_base;
    return (int)total;
}

template <int kMode>
cudaError_t launch_group_t(const void *dev_base, int count, int total_tiles, int *err, cudaStream_t s) {
    using C = Cfg<kMode, false>;
    static std::atomic<bool> attr[64];   // per device, set once; atomic: host threads may launch concurrently
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<kMode, false, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    const char *b = (const char *)dev_base;
    TcGemmArgs g{};
    g.n = kBM;
    g.ldp = 64;
    g.err = err;
    g.gmaps = b;
    g.gargs = reinterpret_cast<const TcGemmArgs *>(b + group_maps_bytes(count));
    g.gstart = reinterpret_cast<const int *>(b + group_maps_bytes(count) + group_args_bytes(count));
    g.gcount = count;
    g.wait_limit = g_debug_wait_limit;
    g.debug_stall = g_debug_stall;
    // the kernel's own maps are not read in a grouped launch; any valid map will do
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    const int64_t S = sm_count();
    const int grid = (int)(total_tiles < S ? total_tiles : S);
    if (grid < 1) return cudaSuccess;
    tc_gemm_kernel<kMode, false, true><<<grid, kThreads, C::kSmem, s>>>(dummy, dummy, dummy, g);
    return cudaGetLastError();
}

}  // namespace

size_t gemm_group_bytes(int count) {
    return group_maps_bytes(count) + group_args_bytes(count) + round_to((size_t)(count + 1) * sizeof(int), 256);
}

int gemm_group_image(const TcGemmArgs *items, int count, int shape, const void *dev_base, std::vector<char> &host) {
    if (!items || count < 1) return -1;
    if (shape == 1) return group_image_t<3>(items, count, dev_base, host);
    if (shape == 2) return group_image_t<4>(items, count, dev_base, host);
    return group_image_t<0>(items, count, dev_base, host);
}

cudaError_t launch_gemm_group(const void *dev_base, int count, int total_tiles, int shape, int *err, cudaStream_t s) {
    if (!dev_base || count < 1 || total_tiles < 0 || ((uintptr_t)dev_base % 256) != 0) return cudaErrorInvalidValue;
    if (shape == 1) return launch_group_t<3>(dev_base, count, total_tiles, err, s);
    if (shape == 2) return launch_group_t<4>(dev_base, count, total_tiles, err, s);
    return launch_group_t<0>(dev_base, count, total_tiles, err, s);
}

cudaError_t launch_gemm_bf16x3(const TcGemmArgs &g, int shape, cudaStream_t s) {
    if (shape == 1) return launch_tc<3>(g, s);
    if (shape == 2) return launch_tc<4>(g, s);
    return launch_tc<0>(g, s);
}
cudaError_t launch_gemm_tf32(const TcGemmArgs &g, cudaStream_t s) { return launch_tc<1>(g, s); }
cudaError_t launch_gemm_bf16x5(const TcGemmArgs &g, cudaStream_t s) {
    if (!g.wide) return cudaErrorInvalidValue;
    return launch_tc<6, true>(g, s);
}
cudaError_t launch_gemm_bf16x4(const TcGemmArgs &g, int shape, cudaStream_t s) {
    if (g.wide) return shape == 2 ? launch_tc<5, true>(g, s) : launch_tc<2, true>(g, s);
    return shape == 2 ? launch_tc<5>(g, s) : launch_tc<2>(g, s);
}

}  // namespace ustat
