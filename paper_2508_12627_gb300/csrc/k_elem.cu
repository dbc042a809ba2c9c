// Tensorization (the paper's Algorithm 1 for the kernel maps), vector operations
// and the final Moebius combination U = sum_pi mu_pi V_pi (Section 3.3, Lemma
// "Decomposition of U-Statistic into V-Statistics"; Algorithm 4).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kcommon.cuh"
#include "kernels.h"
#include "kmath.cuh"
#include "../../include/ustat.h"

namespace ustat {

namespace {

// Error-word bit of a non-finite input (bit 0 is a bounded wait that gave up).
constexpr int kErrNonfinite = kErrWordNonfinite;

// Records a non-finite input value in the error word.
__device__ __forceinline__ void flag_nonfinite(bool bad, int *err) {
    if (bad && err) atomicOr(err, kErrNonfinite);
}

template <typename T>
__global__ void xconvert_kernel(const void *X, int x_dtype, int64_t total, T *out, int *err) {
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        double v = x_dtype == 0 ? ((const double *)X)[t] : (double)((const float *)X)[t];
        bad |= !isfinite(v);
        out[t] = (T)v;
    }
    flag_nonfinite(bad, err);
}

// exp(z) in float32 arithmetic with only one rounding that matters: the result is
// within ~0.6 ulp of e^z and its rounding errors are symmetric (no mean bias), so
// the n^2 kernel entries do not shift a V-statistic systematically.
// Method: Cody-Waite reduction z = k ln2 + f with ln2 = L1 + L2 (L1 = 45426 / 2^16,
// so k L1 is exact), |f| <= ln2 / 2; e^f = 1 + f + f^2 (1/2! + f/3! + ... + f^6/8!)
// (Taylor, truncation error below 2^-32); 1 + f is summed as a double-float and the
// final sum rounded once; e^z = 2^k e^f by exponent arithmetic.
__device__ __forceinline__ float exp_unbiased(float z) {
    if (z < -87.0f) return 0.0f;
    const float k = rintf(z * 1.44269504088896341f);
    const float L1 = 0.693145751953125f;           // 45426 / 65536
    const float L2 = 1.42860682030941723212e-6f;    // ln 2 - L1
    const float fh = fmaf(-k, L1, z);               // exact
    const float fl = -k * L2;
    const float f = fh + fl;
    float q = 1.0f / 40320.0f;
    q = fmaf(q, f, 1.0f / 5040.0f);
    q = fmaf(q, f, 1.0f / 720.0f);
    q = fmaf(q, f, 1.0f / 120.0f);
    q = fmaf(q, f, 1.0f / 24.0f);
    q = fmaf(q, f, 1.0f / 6.0f);
    q = fmaf(q, f, 0.5f);
    q = q * f * f;
    const float sh = 1.0f + fh;                     // Fast2Sum (|1| >= |fh|)
    const float sl = fh - (sh - 1.0f);
    const float y = sh + ((sl + fl) + q);
    const int ki = (int)k;
    return y * __int_as_float((ki + 127) << 23);    // 2^k, k >= -126 here
}

// One 64 x 64 tile of K per block, 16 x 16 threads, 4 x 4 outputs per thread
// (rows ty + 16 r, cols tx + 16 c).  X rows of both tile sides go through shared
// memory in chunks of 32 coordinates.  Float32 version: the squared distance is
// summed in float32 (its rounding errors are symmetric), the exponential is
// exp_unbiased, and the linear kernel's dot product is accumulated as a
// double-float (TwoProd by FMA, TwoSum) and rounded once.
// With a float64 K (TO = double, the float64-storage modes, linear kernel of a
// float32 X): the double-float dot product, exact products and a compensated
// sum, goes to float64 unrounded and is divided in float64.
template <typename TO>
__global__ void __launch_bounds__(256) kbuild_f32_kernel(int kind, float inv_param, const float *__restrict__ X,
                                                         int64_t n, int d, int zero_diag, TO *__restrict__ K,
                                                         double inv_param_d = 0.0) {
    __shared__ float xi[64][33];
    __shared__ float xj[64][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t i0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 64;
    float acc[4][4], lo[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = lo[r][c] = 0.f;
    const int tid = ty * 16 + tx;
    for (int k0 = 0; k0 < d; k0 += 32) {
        for (int e = tid; e < 64 * 32; e += 256) {
            int rr = e / 32, kk = e % 32;
            int64_t gi = i0 + rr, gj = j0 + rr;
            xi[rr][kk] = (gi < n && k0 + kk < d) ? X[gi * d + k0 + kk] : 0.f;
            xj[rr][kk] = (gj < n && k0 + kk < d) ? X[gj * d + k0 + kk] : 0.f;
        }
        __syncthreads();
        const int kmax = min(32, d - k0);
        for (int kk = 0; kk < kmax; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = xi[ty + 16 * r][kk];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = xj[tx + 16 * c][kk];
            if (kind == USTAT_RBF) {
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float df = a[r] - b[c];
                        acc[r][c] = fmaf(df, df, acc[r][c]);
                    }
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float p = a[r] * b[c];
                        const float pe = fmaf(a[r], b[c], -p);
                        const float t = acc[r][c] + p;
                        const float bp = t - acc[r][c];
                        const float se = (acc[r][c] - (t - bp)) + (p - bp);
                        acc[r][c] = t;
                        lo[r][c] += se + pe;
                    }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int64_t gi = i0 + ty + 16 * r;
        if (gi >= n) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int64_t gj = j0 + tx + 16 * c;
            if (gj >= n) continue;
            TO v;
            if constexpr (sizeof(TO) == 8) {
                v = ((double)acc[r][c] + (double)lo[r][c]) * inv_param_d;
            } else if (kind == USTAT_RBF) {
                v = (gi == gj) ? 1.0f : exp_unbiased(-acc[r][c] * inv_param);
            } else {
                const float s = acc[r][c] + lo[r][c];
                v = s * inv_param;
            }
            if (zero_diag && gi == gj) v = TO(0);
            K[gi * n + gj] = v;
        }
    }
}

// RBF kernel matrix in float32, fused with its split into bf16 fixed-point
// slices (the row scale is known: entries lie in (0, 1], so every row scale is
// 1) and with up to kRbfMaxRed reductions of its entrywise powers (a full sum
// sum_ij K_ij^p into a float64 scalar, or row sums sum_j K_ij^p into a float64
// vector).  One block per 128 x 128 tile on or above the diagonal.  Each thread
// owns rows {4 ty + i, 64 + 4 ty + i} and columns {4 tx + j, 64 + 4 tx + j}
// (i, j < 4), so it writes the tile with 16-byte row stores and, off the
// diagonal, the mirror tile with 16-byte stores of its column quadruples; K is
// exactly symmetric because (x_i - x_j)^2 = (x_j - x_i)^2 in every rounding.
// The squared distance is a sum of squared differences (no Gram form: it would
// cancel), the exponential exp_unbiased's steps, the diagonal exactly 1 (0 in
// the sparsified mode).  The arithmetic runs on pairs of float32 with the
// packed .f32x2 instructions (the same IEEE operations per lane, half the
// instructions); the kernel is bound by instruction issue otherwise.
// slices == nullptr: K only.
constexpr int kRbfT = 128;
constexpr int kRbfMaxRed = 4;
struct RbfRed {
    int pow;        // 1..4
    int vec;        // 1: out[i] += sum_j K_ij^pow; 0: out[0] += sum_ij K_ij^pow
    double *out;
};
struct RbfArgs {
    const float *X;          // float32 X, or
    const double *Xd;        // float64 X, rounded to float32 as it is staged (no conversion pass)
    int xvec;                // d % 4 == 0 and X 16-byte aligned: vector loads of X
    int64_t n;
    int d;
    float inv_h;
    int zero_diag;
    float *K;
    __nv_bfloat16 *slices;   // [planes][n][ldp] or null
    int64_t ldp;
    int lead_bits, planes;
    float *scales;
    int nred;
    RbfRed red[kRbfMaxRed];
    int upper_only;   // K itself is read only on and above the diagonal: no mirror stores of K
    int *err;         // error word: the diagonal tiles flag a non-finite X
};

// one row of a thread's entries (four pairs); out of line with the four pairs
// interleaved, so that the kernel's code stays small while each call still has
// four independent dependency chains
struct F2Row {
    f32x2 v[4];
};
__device__ __noinline__ F2Row f2_rbf_row(F2Row d2, float inv_h) {
    F2Row r;
#pragma unroll
    for (int h = 0; h < 4; ++h) r.v[h] = f2_rbf(d2.v[h], inv_h);
    return r;
}

__device__ __forceinline__ int rbf_row(int a, int ty) { return 4 * ty + (a & 3) + 64 * (a >> 2); }

// eight entries of row gr (columns gc..gc+3 and gc+64..gc+67) of K and of its
// digit planes.  Digit p of y = K * 2^w is y_p rounded to a multiple of 2^-8p by
// adding and subtracting 1.5 * 2^(23 - 8p) (round to nearest even, exact for
// |y_p| < 2^(22 - 8p)); the remainder y_{p+1} = y_p - digit is exact.  Out of
// line: the kernel calls it 16 times, and inlined copies outgrew the
// instruction cache.
// (half: the column offset of the second quadruple, 64 for 128-wide tiles and 32
// for 64-wide ones; nhalf = 1 stores the first quadruple only)
template <int nhalf = 2>
__device__ __noinline__ void rbf_store_row(float *K, __nv_bfloat16 *slices, int64_t n, int64_t ldp, int planes,
                                           float lead_scale, int64_t gr, int64_t gc, F2Row v, int half = 64) {
    float *krow = K ? K + gr * n : nullptr;
    const bool vec4 = (n % 4) == 0;
#pragma unroll
    for (int hh = 0; hh < 2 && krow; ++hh) {
        if (hh >= nhalf) break;
        const int64_t c = gc + half * hh;
        float e[4];
        f2_unpack(v.v[2 * hh], e[0], e[1]);
        f2_unpack(v.v[2 * hh + 1], e[2], e[3]);
        if (vec4 && c + 3 < n) {
            *reinterpret_cast<float4 *>(krow + c) = make_float4(e[0], e[1], e[2], e[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (c + q < n) krow[c + q] = e[q];
        }
    }
    if (!slices) return;
    const f32x2 ls = f2_splat(lead_scale);
    f32x2 y[4];
#pragma unroll
    for (int h = 0; h < 2 * nhalf; ++h) y[h] = f2_mul(v.v[h], ls);   // row scale 1: |y| <= 2^w, exact
    const int64_t plane = n * ldp;
    __nv_bfloat16 *srow = slices + gr * ldp + gc;
    float magic = 12582912.0f;   // 1.5 * 2^23
    for (int p = 0; p < planes; ++p) {
        const f32x2 mg = f2_splat(magic);
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 2 * nhalf; ++h) {
            const f32x2 dgt = f2_sub(f2_add(y[h], mg), mg);
            y[h] = f2_sub(y[h], dgt);
            float d0, d1;
            f2_unpack(dgt, d0, d1);
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(d0, d1);
            w[h] = *reinterpret_cast<const uint32_t *>(&b2);
        }
        __nv_bfloat16 *dst = srow + p * plane;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            if (hh >= nhalf) break;
            const int64_t c = gc + half * hh;
            if (c + 3 < ldp) {
                *reinterpret_cast<uint2 *>(dst + half * hh) = make_uint2(w[2 * hh], w[2 * hh + 1]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c + q < ldp)
                        dst[half * hh + q] = __ushort_as_bfloat16((uint16_t)(w[2 * hh + (q >> 1)] >> (16 * (q & 1))));
            }
        }
        magic *= (1.0f / 256.0f);
    }
}

__global__ void __launch_bounds__(256, 2) kbuild_rbf_tile_kernel(RbfArgs g) {
    // coordinates k of the tile's rows: xa[k][r] = (x, x) pairs for the rows,
    // xb[k][r] for the columns; xa is reused by the reductions
    __shared__ __align__(16) float2 xa[32][kRbfT];
    __shared__ __align__(16) float xb[32][kRbfT];
    __shared__ double dred[8];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, warp = tid >> 5;
    const int64_t n = g.n;
    const int T = (int)((g.ldp + kRbfT - 1) / kRbfT);
    // upper-triangle tile t -> (tm, tn), row-major: row r starts at r T - r (r - 1) / 2
    const int t = blockIdx.x;
    const double bq = 2.0 * T + 1.0;
    int tm = (int)((bq - sqrt(bq * bq - 8.0 * t)) * 0.5);
    if (tm < 0) tm = 0;
    while (tm > 0 && tm * T - tm * (tm - 1) / 2 > t) --tm;
    while (tm + 1 < T && (tm + 1) * T - (tm + 1) * tm / 2 <= t) ++tm;
    const int tn = tm + (t - (tm * T - tm * (tm - 1) / 2));
    const int64_t i0 = (int64_t)tm * kRbfT, j0 = (int64_t)tn * kRbfT;
    const bool diag_tile = tm == tn;

    // acc[a][h]: row a, columns (2h, 2h + 1) of the thread's eight
    f32x2 acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int h = 0; h < 4; ++h) acc[a][h] = f2_splat(0.f);
    const bool xvec = g.xvec != 0;
    // every row of X is staged once as the row side of its diagonal tile: that
    // staging also checks it for non-finite values
    bool bad = false;
    for (int k0 = 0; k0 < g.d; k0 += 32) {
        __syncthreads();
        // stage rows i0.. and j0.., 32 coordinates, transposed (consecutive lanes:
        // consecutive rows, so the shared-memory writes do not conflict)
        for (int e = tid; e < 2 * kRbfT * 8; e += 256) {
            const int opnd = e >> 10, row = e & (kRbfT - 1), kq = (e >> 7) & 7;
            const bool check = diag_tile && opnd == 0;
            const int64_t gr = (opnd ? j0 : i0) + row;
            const int k = k0 + 4 * kq;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gr < n && k < g.d) {
                if (g.Xd) {
                    const double *src = g.Xd + gr * g.d + k;
                    if (xvec) {
                        const double2 p0 = *reinterpret_cast<const double2 *>(src);
                        const double2 p1 = *reinterpret_cast<const double2 *>(src + 2);
                        v = make_float4((float)p0.x, (float)p0.y, (float)p1.x, (float)p1.y);
                        if (check) bad |= !(isfinite(p0.x) && isfinite(p0.y) && isfinite(p1.x) && isfinite(p1.y));
                    } else {
                        double q[4] = {src[0], 0.0, 0.0, 0.0};
                        if (k + 1 < g.d) q[1] = src[1];
                        if (k + 2 < g.d) q[2] = src[2];
                        if (k + 3 < g.d) q[3] = src[3];
                        v = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
                        if (check) bad |= !(isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]));
                    }
                } else {
                    const float *src = g.X + gr * g.d + k;
                    if (xvec) {
                        v = *reinterpret_cast<const float4 *>(src);
                    } else {
                        v.x = src[0];
                        if (k + 1 < g.d) v.y = src[1];
                        if (k + 2 < g.d) v.z = src[2];
                        if (k + 3 < g.d) v.w = src[3];
                    }
                    if (check) bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
                }
            }
            if (opnd == 0) {
                xa[4 * kq + 0][row] = make_float2(v.x, v.x);
                xa[4 * kq + 1][row] = make_float2(v.y, v.y);
                xa[4 * kq + 2][row] = make_float2(v.z, v.z);
                xa[4 * kq + 3][row] = make_float2(v.w, v.w);
            } else {
                xb[4 * kq + 0][row] = v.x;
                xb[4 * kq + 1][row] = v.y;
                xb[4 * kq + 2][row] = v.z;
                xb[4 * kq + 3][row] = v.w;
            }
        }
        __syncthreads();
        const int kmax = min(32, g.d - k0);
        for (int kk = 0; kk < kmax; ++kk) {
            f32x2 av[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = (q & 1) * 2 + (q >> 1) * 64 + 4 * ty;
                const ulonglong2 pr = *reinterpret_cast<const ulonglong2 *>(&xa[kk][r]);
                av[(q >> 1) * 4 + (q & 1) * 2] = pr.x;
                av[(q >> 1) * 4 + (q & 1) * 2 + 1] = pr.y;
            }
            const ulonglong2 b0 = *reinterpret_cast<const ulonglong2 *>(&xb[kk][4 * tx]);
            const ulonglong2 b1 = *reinterpret_cast<const ulonglong2 *>(&xb[kk][64 + 4 * tx]);
            const f32x2 bv[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
            for (int a = 0; a < 8; ++a) {
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const f32x2 df = f2_sub(av[a], bv[h]);
                    acc[a][h] = f2_fma(df, df, acc[a][h]);
                }
            }
        }
    }
    if (diag_tile) flag_nonfinite(bad, g.err);
    // entries: exp off the diagonal, the diagonal exactly, zero in the padding
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        F2Row d2;
#pragma unroll
        for (int h = 0; h < 4; ++h) d2.v[h] = acc[a][h];
        const F2Row e = f2_rbf_row(d2, g.inv_h);
#pragma unroll
        for (int h = 0; h < 4; ++h) acc[a][h] = e.v[h];
    }
    if (diag_tile || i0 + kRbfT > n || j0 + kRbfT > n) {
        const float dv = g.zero_diag ? 0.f : 1.f;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int64_t gi = i0 + rbf_row(a, ty);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                float e0, e1;
                f2_unpack(acc[a][h], e0, e1);
                const int64_t gj0 = j0 + rbf_row(2 * h, tx), gj1 = j0 + rbf_row(2 * h + 1, tx);
                if (gi == gj0) e0 = dv;
                if (gi == gj1) e1 = dv;
                if (gi >= n || gj0 >= n) e0 = 0.f;
                if (gi >= n || gj1 >= n) e1 = 0.f;
                acc[a][h] = f2_pack(e0, e1);
            }
        }
    }

    // fused reductions of K^p (block-uniform control flow)
    if (g.nred > 0) {
        __syncthreads();   // the staging buffer becomes the column-partial buffer
        float *colpart = reinterpret_cast<float *>(&xa[0][0]);   // [8 warps][128]
        for (int q = 0; q < g.nred; ++q) {
            const int p = g.red[q].pow;
            double *out = g.red[q].out;
            f32x2 cq[4];
            float rp[8];
#pragma unroll
            for (int h = 0; h < 4; ++h) cq[h] = f2_splat(0.f);
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                f32x2 w[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) w[h] = acc[a][h];
                for (int e = 1; e < p; ++e) {
#pragma unroll
                    for (int h = 0; h < 4; ++h) w[h] = f2_mul(w[h], acc[a][h]);
                }
                float r0, r1;
                f2_unpack(f2_add(f2_add(w[0], w[1]), f2_add(w[2], w[3])), r0, r1);
                rp[a] = r0 + r1;
#pragma unroll
                for (int h = 0; h < 4; ++h) cq[h] = f2_add(cq[h], w[h]);
            }
            if (g.red[q].vec) {
                // rows of this tile: reduce over the 16 lanes of one ty
#pragma unroll
                for (int a = 0; a < 8; ++a) {
#pragma unroll
                    for (int o = 8; o > 0; o >>= 1) rp[a] += __shfl_xor_sync(0xffffffffu, rp[a], o);
                }
                if (tx == 0) {
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        const int64_t gi = i0 + rbf_row(a, ty);
                        if (gi < n) atomicAdd(out + gi, (double)rp[a]);
                    }
                }
                if (!diag_tile) {
                    // rows of the mirror tile = columns of this one
                    float cv[8];
#pragma unroll
                    for (int h = 0; h < 4; ++h) f2_unpack(cq[h], cv[2 * h], cv[2 * h + 1]);
#pragma unroll
                    for (int c = 0; c < 8; ++c) cv[c] += __shfl_xor_sync(0xffffffffu, cv[c], 16);
                    if (lane < 16) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) colpart[warp * kRbfT + rbf_row(c, tx)] = cv[c];
                    }
                    __syncthreads();
                    if (tid < kRbfT && j0 + tid < n) {
                        float s = 0.f;
#pragma unroll
                        for (int w = 0; w < 8; ++w) s += colpart[w * kRbfT + tid];
                        atomicAdd(out + j0 + tid, (double)s);
                    }
                    __syncthreads();
                }
            } else {
                double s = (double)(((rp[0] + rp[1]) + (rp[2] + rp[3])) + ((rp[4] + rp[5]) + (rp[6] + rp[7])));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) dred[warp] = s;
                __syncthreads();
                if (tid == 0) {
                    double tsum = 0.0;
#pragma unroll
                    for (int w = 0; w < 8; ++w) tsum += dred[w];
                    atomicAdd(out, diag_tile ? tsum : 2.0 * tsum);
                }
                __syncthreads();
            }
        }
    }

    const float lead_scale = __int_as_float((127 + g.lead_bits) << 23);   // 2^w
    float *K = g.K;
    __nv_bfloat16 *slices = g.slices;
    const int64_t ldp = g.ldp;
    const int planes = g.planes;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int64_t gr = i0 + rbf_row(a, ty);
        if (gr >= n) continue;
        F2Row v;
#pragma unroll
        for (int h = 0; h < 4; ++h) v.v[h] = acc[a][h];
        rbf_store_row(K, slices, n, ldp, planes, lead_scale, gr, j0 + 4 * tx, v);
    }
    if (!diag_tile) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float c0[8], c1[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) f2_unpack(acc[a][h], c0[a], c1[a]);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const float *cv = s ? c1 : c0;
                const int64_t gr = j0 + rbf_row(2 * h + s, tx);
                if (gr >= n) continue;
                F2Row v;
#pragma unroll
                for (int q = 0; q < 4; ++q) v.v[q] = f2_pack(cv[2 * q], cv[2 * q + 1]);
                rbf_store_row(g.upper_only ? nullptr : K, slices, n, ldp, planes, lead_scale, gr, i0 + 4 * ty, v);
            }
        }
    }
    if (g.scales && diag_tile && tid < kRbfT && i0 + tid < n) g.scales[i0 + tid] = 1.f;
}


// The same build on 64 x 64 tiles with 128 threads (4 x 8 entries per thread):
// half the registers per thread, so four times as many warps per SM fit, for
// the latency of the epilogue's dependent chains.  Thread (ty, tx), ty < 16,
// tx < 8, owns rows 4 ty + i and columns {4 tx + j, 32 + 4 tx + j}.
constexpr int kRbfT64 = 64;
__global__ void __launch_bounds__(128, 8) kbuild_rbf_tile64_kernel(RbfArgs g) {
    __shared__ __align__(16) float2 xa[32][kRbfT64];
    __shared__ __align__(16) float xb[32][kRbfT64];
    __shared__ double dred[4];
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3, lane = tid & 31, warp = tid >> 5;
    const int64_t n = g.n;
    const int T = (int)((g.ldp + kRbfT64 - 1) / kRbfT64);
    const int t = blockIdx.x;
    const double bq = 2.0 * T + 1.0;
    int tm = (int)((bq - sqrt(bq * bq - 8.0 * t)) * 0.5);
    if (tm < 0) tm = 0;
    while (tm > 0 && tm * T - tm * (tm - 1) / 2 > t) --tm;
    while (tm + 1 < T && (tm + 1) * T - (tm + 1) * tm / 2 <= t) ++tm;
    const int tn = tm + (t - (tm * T - tm * (tm - 1) / 2));
    const int64_t i0 = (int64_t)tm * kRbfT64, j0 = (int64_t)tn * kRbfT64;
    const bool diag_tile = tm == tn;

    f32x2 acc[4][4];   // [row i][column pair h]: columns (2h, 2h + 1) of {4 tx .., 32 + 4 tx ..}
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int h = 0; h < 4; ++h) acc[a][h] = f2_splat(0.f);
    const bool xvec = g.xvec != 0;
    bool bad = false;   // as in the 128-tile form: diagonal tiles check X
    for (int k0 = 0; k0 < g.d; k0 += 32) {
        __syncthreads();
        for (int e = tid; e < 2 * kRbfT64 * 8; e += 128) {
            const int opnd = e >> 9, row = e & (kRbfT64 - 1), kq = (e >> 6) & 7;
            const bool check = diag_tile && opnd == 0;
            const int64_t gr = (opnd ? j0 : i0) + row;
            const int k = k0 + 4 * kq;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gr < n && k < g.d) {
                if (g.Xd) {
                    const double *src = g.Xd + gr * g.d + k;
                    if (xvec) {
                        const double2 p0 = *reinterpret_cast<const double2 *>(src);
                        const double2 p1 = *reinterpret_cast<const double2 *>(src + 2);
                        v = make_float4((float)p0.x, (float)p0.y, (float)p1.x, (float)p1.y);
                        if (check) bad |= !(isfinite(p0.x) && isfinite(p0.y) && isfinite(p1.x) && isfinite(p1.y));
                    } else {
                        double q[4] = {src[0], 0.0, 0.0, 0.0};
                        if (k + 1 < g.d) q[1] = src[1];
                        if (k + 2 < g.d) q[2] = src[2];
                        if (k + 3 < g.d) q[3] = src[3];
                        v = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
                        if (check) bad |= !(isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]));
                    }
                } else {
                    const float *src = g.X + gr * g.d + k;
                    if (xvec) {
                        v = *reinterpret_cast<const float4 *>(src);
                    } else {
                        v.x = src[0];
                        if (k + 1 < g.d) v.y = src[1];
                        if (k + 2 < g.d) v.z = src[2];
                        if (k + 3 < g.d) v.w = src[3];
                    }
                    if (check) bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
                }
            }
            if (opnd == 0) {
                xa[4 * kq + 0][row] = make_float2(v.x, v.x);
                xa[4 * kq + 1][row] = make_float2(v.y, v.y);
                xa[4 * kq + 2][row] = make_float2(v.z, v.z);
                xa[4 * kq + 3][row] = make_float2(v.w, v.w);
            } else {
                xb[4 * kq + 0][row] = v.x;
                xb[4 * kq + 1][row] = v.y;
                xb[4 * kq + 2][row] = v.z;
                xb[4 * kq + 3][row] = v.w;
            }
        }
        __syncthreads();
        const int kmax = min(32, g.d - k0);
        for (int kk = 0; kk < kmax; ++kk) {
            const ulonglong2 a01 = *reinterpret_cast<const ulonglong2 *>(&xa[kk][4 * ty]);
            const ulonglong2 a23 = *reinterpret_cast<const ulonglong2 *>(&xa[kk][4 * ty + 2]);
            const f32x2 av[4] = {a01.x, a01.y, a23.x, a23.y};
            const ulonglong2 b0 = *reinterpret_cast<const ulonglong2 *>(&xb[kk][4 * tx]);
            const ulonglong2 b1 = *reinterpret_cast<const ulonglong2 *>(&xb[kk][32 + 4 * tx]);
            const f32x2 bv[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const f32x2 df = f2_sub(av[a], bv[h]);
                    acc[a][h] = f2_fma(df, df, acc[a][h]);
                }
        }
    }
    if (diag_tile) flag_nonfinite(bad, g.err);
    auto colof = [&](int c) { return 4 * tx + (c & 3) + 32 * (c >> 2); };   // c < 8
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        F2Row d2;
#pragma unroll
        for (int h = 0; h < 4; ++h) d2.v[h] = acc[a][h];
        const F2Row e = f2_rbf_row(d2, g.inv_h);
#pragma unroll
        for (int h = 0; h < 4; ++h) acc[a][h] = e.v[h];
    }
    if (diag_tile || i0 + kRbfT64 > n || j0 + kRbfT64 > n) {
        const float dv = g.zero_diag ? 0.f : 1.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t gi = i0 + 4 * ty + a;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                float e0, e1;
                f2_unpack(acc[a][h], e0, e1);
                const int64_t gj0 = j0 + colof(2 * h), gj1 = j0 + colof(2 * h + 1);
                if (gi == gj0) e0 = dv;
                if (gi == gj1) e1 = dv;
                if (gi >= n || gj0 >= n) e0 = 0.f;
                if (gi >= n || gj1 >= n) e1 = 0.f;
                acc[a][h] = f2_pack(e0, e1);
            }
        }
    }

    if (g.nred > 0) {
        __syncthreads();
        float *colpart = reinterpret_cast<float *>(&xa[0][0]);   // [4 warps][64]
        for (int q = 0; q < g.nred; ++q) {
            const int p = g.red[q].pow;
            double *out = g.red[q].out;
            f32x2 cq[4];
            float rp[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) cq[h] = f2_splat(0.f);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                f32x2 w[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) w[h] = acc[a][h];
                for (int e = 1; e < p; ++e) {
#pragma unroll
                    for (int h = 0; h < 4; ++h) w[h] = f2_mul(w[h], acc[a][h]);
                }
                float r0, r1;
                f2_unpack(f2_add(f2_add(w[0], w[1]), f2_add(w[2], w[3])), r0, r1);
                rp[a] = r0 + r1;
#pragma unroll
                for (int h = 0; h < 4; ++h) cq[h] = f2_add(cq[h], w[h]);
            }
            if (g.red[q].vec) {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
#pragma unroll
                    for (int o = 4; o > 0; o >>= 1) rp[a] += __shfl_xor_sync(0xffffffffu, rp[a], o);
                }
                if (tx == 0) {
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int64_t gi = i0 + 4 * ty + a;
                        if (gi < n) atomicAdd(out + gi, (double)rp[a]);
                    }
                }
                if (!diag_tile) {
                    float cv[8];
#pragma unroll
                    for (int h = 0; h < 4; ++h) f2_unpack(cq[h], cv[2 * h], cv[2 * h + 1]);
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        cv[c] += __shfl_xor_sync(0xffffffffu, cv[c], 8);
                        cv[c] += __shfl_xor_sync(0xffffffffu, cv[c], 16);
                    }
                    if (lane < 8) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) colpart[warp * kRbfT64 + colof(c)] = cv[c];
                    }
                    __syncthreads();
                    if (tid < kRbfT64 && j0 + tid < n) {
                        const float sum = (colpart[tid] + colpart[kRbfT64 + tid]) +
                                          (colpart[2 * kRbfT64 + tid] + colpart[3 * kRbfT64 + tid]);
                        atomicAdd(out + j0 + tid, (double)sum);
                    }
                    __syncthreads();
                }
            } else {
                double sd = (double)((rp[0] + rp[1]) + (rp[2] + rp[3]));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
                if (lane == 0) dred[warp] = sd;
                __syncthreads();
                if (tid == 0) {
                    const double tsum = (dred[0] + dred[1]) + (dred[2] + dred[3]);
                    atomicAdd(out, diag_tile ? tsum : 2.0 * tsum);
                }
                __syncthreads();
            }
        }
    }

    const float lead_scale = __int_as_float((127 + g.lead_bits) << 23);   // 2^w
    float *K = g.K;
    __nv_bfloat16 *slices = g.slices;
    const int64_t ldp = g.ldp;
    const int planes = g.planes;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t gr = i0 + 4 * ty + a;
        if (gr >= n) continue;
        F2Row v;
#pragma unroll
        for (int h = 0; h < 4; ++h) v.v[h] = acc[a][h];
        rbf_store_row<2>(K, slices, n, ldp, planes, lead_scale, gr, j0 + 4 * tx, v, 32);
    }
    // K below the diagonal is skipped only where no reader needs it: the readers
    // of an upper-only K are symmetric GEMMs with 128-row tiles, whose diagonal
    // tiles also read the lower 64 x 64 tile of each diagonal 128 x 128 block
    const bool mirror_k = !g.upper_only || (tn == tm + 1 && (tm & 1) == 0);
    if (!diag_tile) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float c0[4], c1[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) f2_unpack(acc[a][h], c0[a], c1[a]);
#pragma unroll
            for (int sdx = 0; sdx < 2; ++sdx) {
                const float *cv = sdx ? c1 : c0;
                const int64_t gr = j0 + colof(2 * h + sdx);
                if (gr >= n) continue;
                F2Row v;
                v.v[0] = f2_pack(cv[0], cv[1]);
                v.v[1] = f2_pack(cv[2], cv[3]);
                v.v[2] = v.v[3] = f2_splat(0.f);
                rbf_store_row<1>(mirror_k ? K : nullptr, slices, n, ldp, planes, lead_scale, gr, i0 + 4 * ty, v, 32);
            }
        }
    }
    if (g.scales && diag_tile && tid < kRbfT64 && i0 + tid < n) g.scales[i0 + tid] = 1.f;
}

// Float64 version (FP64 mode).
template <typename T>
__global__ void __launch_bounds__(256) kbuild_kernel(int kind, T inv_param, const T *__restrict__ X,
                                                     int64_t n, int d, int zero_diag, T *__restrict__ K) {
    __shared__ T xi[64][33];
    __shared__ T xj[64][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t i0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 64;
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0;
    const int tid = ty * 16 + tx;
    for (int k0 = 0; k0 < d; k0 += 32) {
        for (int e = tid; e < 64 * 32; e += 256) {
            int rr = e / 32, kk = e % 32;
            int64_t gi = i0 + rr, gj = j0 + rr;
            xi[rr][kk] = (gi < n && k0 + kk < d) ? X[gi * d + k0 + kk] : T(0);
            xj[rr][kk] = (gj < n && k0 + kk < d) ? X[gj * d + k0 + kk] : T(0);
        }
        __syncthreads();
        const int kmax = min(32, d - k0);
        for (int kk = 0; kk < kmax; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = xi[ty + 16 * r][kk];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = xj[tx + 16 * c][kk];
            if (kind == USTAT_RBF) {
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        T df = a[r] - b[c];
                        acc[r][c] = fma(df, df, acc[r][c]);
                    }
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int64_t gi = i0 + ty + 16 * r;
        if (gi >= n) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int64_t gj = j0 + tx + 16 * c;
            if (gj >= n) continue;
            T v = (kind == USTAT_RBF) ? exp(-acc[r][c] * inv_param) : acc[r][c] * inv_param;
            if (zero_diag && gi == gj) v = 0;
            K[gi * n + gj] = v;
        }
    }
}

// A caller matrix as the storage type; with `complement`, the factor 1 - A (the
// motif kernels' non-edge factor B = 1 - A, Section 4.2).
template <typename T>
__global__ void loadmat_kernel(const double *src, int64_t n, int zero_diag, int complement, T *dst, int *err) {
    const int64_t total = n * n;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double x = src[t];
        bad |= !isfinite(x);
        T v = (T)(complement ? 1.0 - x : x);
        if (zero_diag && (t / n) == (t % n)) v = 0;
        dst[t] = v;
    }
    flag_nonfinite(bad, err);
}

__global__ void unary_tanh_kernel(const void *X, int x_dtype, int64_t n, int d, const double *w, double *out,
                                  int *err) {
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            double x = x_dtype == 0 ? ((const double *)X)[i * d + k] : (double)((const float *)X)[i * d + k];
            s = fma(x, w[k], s);
        }
        bad |= !isfinite(s);   // a non-finite x or w makes the dot product non-finite
        out[i] = tanh(s);
    }
    flag_nonfinite(bad, err);
}

__global__ void copyvec_kernel(const double *src, int64_t n, double *dst, int *err) {
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        bad |= !isfinite(src[i]);
        dst[i] = src[i];
    }
    flag_nonfinite(bad, err);
}

template <typename T>
__global__ void diag_kernel(const T *M, int64_t n, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)M[i * n + i];
}

// Pairwise factors built from caller data on 32 x 32 tiles (32 x 8 threads, four
// entries per thread), float64 arithmetic, rows of both operands staged in shared
// memory in chunks of 64 coordinates:
//   PAIRS_LOWRANK: F(i, j) = sum_k P(i, k) Q(j, k), data = [P | Q] (n x 2r): the
//     HOIF factors g = Psi Psi' and f = Psi Theta' of Section 4.1 from the n x r
//     dictionary terms;
//   PAIRS_DIST: F(i, j) = ||y_i - y_j|| from the coordinate differences, data = Y
//     (n x r): the distance matrices of dCov (Section 4.3), diagonal exactly 0.
//   PAIRS_GRAM: F(i, j) = sum_k P(i, k) P(j, k), data = P (n x r); symmetric.
enum { PAIRS_LOWRANK = 0, PAIRS_DIST = 1, PAIRS_GRAM = 2 };
template <typename T>
__global__ void __launch_bounds__(256) pairs_kernel(int mode, const double *__restrict__ D, int r, int64_t n,
                                                    int zero_diag, T *__restrict__ dst, int *err) {
    __shared__ double as[32][65], bs[32][65];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
    const int ld = mode == PAIRS_LOWRANK ? 2 * r : r;
    const int boff = mode == PAIRS_LOWRANK ? r : 0;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    for (int k0 = 0; k0 < r; k0 += 64) {
        const int kc = min(64, r - k0);
        __syncthreads();
        for (int e = ty * 32 + tx; e < 32 * kc; e += 256) {
            const int row = e / kc, k = e - row * kc;
            const double av = i0 + row < n ? D[(i0 + row) * ld + k0 + k] : 0.0;
            const double bv = j0 + row < n ? D[(j0 + row) * ld + boff + k0 + k] : 0.0;
            bad |= !isfinite(av) || !isfinite(bv);
            as[row][k] = av;
            bs[row][k] = bv;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int rr = ty + 8 * q;
            double a = acc[q];
            if (mode != PAIRS_DIST) {
                for (int k = 0; k < kc; ++k) a = fma(as[rr][k], bs[tx][k], a);
            } else {
                for (int k = 0; k < kc; ++k) {
                    const double df = as[rr][k] - bs[tx][k];
                    a = fma(df, df, a);
                }
            }
            acc[q] = a;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = i0 + ty + 8 * q, j = j0 + tx;
        if (i >= n || j >= n) continue;
        double v = mode == PAIRS_DIST ? sqrt(acc[q]) : acc[q];
        if (i == j && (zero_diag || mode == PAIRS_DIST)) v = 0.0;
        dst[i * n + j] = (T)v;
    }
    flag_nonfinite(bad, err);
}

// Diagonal of a factor from its own data, in float64: x_i . x_i / param for the
// linear kernel (X as given, float64 or float32), M[i][i] for a caller matrix;
// 0 in the sparsified mode.  The stored working-precision matrix would round
// every entry to float32 first, and a partition whose blocks merge all indices
// multiplies several diagonal entries per term.
__global__ void factor_diag_kernel(int kind, double inv_param, const void *X, int x_dtype, int d,
                                   const double *Mc, int64_t n, int zero_diag, double *out, int r) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (!zero_diag) {
            if (kind == USTAT_LINEAR) {
                for (int k = 0; k < d; ++k) {
                    const double x = x_dtype == 0 ? ((const double *)X)[i * d + k] : (double)((const float *)X)[i * d + k];
                    v = fma(x, x, v);
                }
                v *= inv_param;
            } else if (kind == USTAT_RBF) {
                v = 1.0;
            } else if (kind == USTAT_LOWRANK) {
                for (int k = 0; k < r; ++k) v = fma(Mc[i * 2 * r + k], Mc[i * 2 * r + r + k], v);
            } else if (kind == USTAT_GRAM) {
                for (int k = 0; k < r; ++k) v = fma(Mc[i * r + k], Mc[i * r + k], v);
            } else if (kind == USTAT_DIST) {
                v = 0.0;
            } else if (kind == USTAT_COMPLEMENT) {
                v = 1.0 - Mc[i * n + i];
            } else {
                v = Mc[i * n + i];
            }
        }
        out[i] = v;
    }
}

__global__ void vmul_kernel(const double *a, const double *b, int64_t n, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] * b[i];
}

__global__ void vsum_kernel(const double *u, int64_t n, double *out) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += u[i];
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

__global__ void vdot_kernel(const double *u, const double *a, int64_t n, double *out) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(u[i], a[i], s);
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

// Neumaier-compensated running sum (float64).
struct Neumaier {
    double s = 0.0, c = 0.0;
    __device__ void add(double x) {
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ double value() const { return s + c; }
};

// V_pi = prod of its scalar slots * n^(free blocks); U_sum = sum_pi mu_pi V_pi;
// U_mean = U_sum / (n)_m.  One block of 256 threads: the partitions' V are formed
// in parallel, each thread sums its mu V terms with Neumaier compensation, and the
// per-thread (sum, compensation) pairs are combined by one thread in a fixed
// order (deterministic).  The table is a kernel parameter sized to the plan.
template <int CAP>
struct CombineTableT {
    int nparts, m;
    CombineEntry e[CAP];
};

// Sum of a and b split into the rounded sum and its exact rounding error (TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <int CAP>
__global__ void __launch_bounds__(32) combine_kernel(const CombineTableT<CAP> tab, const double *scal,
                                                     const int *err, int64_t n, double *U_out, double *V_out) {
    // one warp: lane l forms V for partitions l, l + 32, ... and sums its mu V
    // terms with Neumaier compensation; the 32 partial sums are then added by a
    // shuffle tree whose rounding errors (TwoSum) are carried separately
    const int lane = threadIdx.x;
    const bool bad = err && *err != 0;
    const double dn = (double)n;
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    Neumaier acc;
    for (int p = lane; p < tab.nparts; p += 32) {
        const CombineEntry en = tab.e[p];
        double v = 0.0;
        if (en.evaluated) {
            double f[kCombineMaxScal];
#pragma unroll
            for (int q = 0; q < kCombineMaxScal; ++q) f[q] = en.sid[q] != 0xffff ? scal[en.sid[q]] : 1.0;
            v = ((f[0] * f[1]) * (f[2] * f[3])) * (f[4] * f[5]);
            for (int q = 0; q < en.nfree; ++q) v *= dn;
        }
        if (bad) v = qnan;
        if (V_out) V_out[p] = v;
        acc.add((double)en.mu * v);
    }
    double s = acc.s, c = acc.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const double c2 = __shfl_xor_sync(0xffffffffu, c, o);
        double t, e;
        two_sum(s, s2, t, e);
        s = t;
        c = c + c2 + e;
    }
    if (lane == 0) {
        double ff = 1.0;
        for (int q = 0; q < tab.m; ++q) ff *= (dn - q);
        const double u = bad ? qnan : s + c;
        U_out[0] = u;
        U_out[1] = u / ff;
    }
}

template <int CAP>
cudaError_t combine_cap(const CombineEntry *entries, int nparts, int m, const double *scal, const int *err,
                        int64_t n, double *U_out, double *V_out, cudaStream_t s) {
    CombineTableT<CAP> tab;
    tab.nparts = nparts;
    tab.m = m;
    for (int p = 0; p < nparts; ++p) tab.e[p] = entries[p];
    combine_kernel<CAP><<<1, 32, 0, s>>>(tab, scal, err, n, U_out, V_out);
    return cudaGetLastError();
}

int grid_for(int64_t total, int threads) {
    int64_t g = (total + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t launch_xconvert(const void *X, int x_dtype, int64_t n, int d, void *Xw, bool fp64, int *err,
                            cudaStream_t s) {
    int64_t total = n * d;
    if (fp64) xconvert_kernel<double><<<grid_for(total, 256), 256, 0, s>>>(X, x_dtype, total, (double *)Xw, err);
    else xconvert_kernel<float><<<grid_for(total, 256), 256, 0, s>>>(X, x_dtype, total, (float *)Xw, err);
    return cudaGetLastError();
}

cudaError_t launch_kbuild(int kind, double param, const void *Xw, bool fp64, int64_t n, int d, int zero_diag,
                          void *K, cudaStream_t s) {
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)((n + 63) / 64)), block(16, 16);
    if (fp64)
        kbuild_kernel<double><<<grid, block, 0, s>>>(kind, 1.0 / param, (const double *)Xw, n, d, zero_diag,
                                                     (double *)K);
    else
        kbuild_f32_kernel<float><<<grid, block, 0, s>>>(kind, (float)(1.0 / param), (const float *)Xw, n, d,
                                                        zero_diag, (float *)K);
    return cudaGetLastError();
}

cudaError_t launch_kbuild_linear_wide(const float *X, int64_t n, int d, double param, int zero_diag, double *K,
                                      cudaStream_t s) {
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)((n + 63) / 64)), block(16, 16);
    kbuild_f32_kernel<double><<<grid, block, 0, s>>>(USTAT_LINEAR, 0.f, X, n, d, zero_diag, K, 1.0 / param);
    return cudaGetLastError();
}

cudaError_t launch_kbuild_rbf(const float *Xw, const double *Xd, int64_t n, int d, double param, int zero_diag,
                              float *K, void *slices, int64_t ldp, int lead_bits, int planes, float *scales, int nred,
                              const int *red_pow, const int *red_vec, double *const *red_out, int upper_only,
                              int tile64, int *err, cudaStream_t s) {
    if (nred < 0 || nred > kRbfMaxRed || planes < 3 || planes > 5 || (!Xw && !Xd)) return cudaErrorInvalidValue;
    const int xvec = (d % 4) == 0 && ((uintptr_t)(Xw ? (const void *)Xw : (const void *)Xd) % 16) == 0;
    RbfArgs g{Xw, Xd, xvec, n, d, (float)(1.0 / param), zero_diag, K, (__nv_bfloat16 *)slices, slices ? ldp : n,
              lead_bits, planes, slices ? scales : nullptr, nred, {}, upper_only, err};
    for (int q = 0; q < nred; ++q) {
        if (red_pow[q] < 1 || red_pow[q] > 4) return cudaErrorInvalidValue;
        g.red[q] = RbfRed{red_pow[q], red_vec[q], red_out[q]};
    }
    if (tile64) {
        const int64_t T = (g.ldp + kRbfT64 - 1) / kRbfT64;
        kbuild_rbf_tile64_kernel<<<(unsigned)(T * (T + 1) / 2), 128, 0, s>>>(g);
    } else {
        const int64_t T = (g.ldp + kRbfT - 1) / kRbfT;
        kbuild_rbf_tile_kernel<<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(g);
    }
    return cudaGetLastError();
}

cudaError_t launch_loadmat(const double *src, int64_t n, bool fp64, int zero_diag, int complement, void *dst,
                           int *err, cudaStream_t s) {
    if (fp64)
        loadmat_kernel<double><<<grid_for(n * n, 256), 256, 0, s>>>(src, n, zero_diag, complement, (double *)dst, err);
    else
        loadmat_kernel<float><<<grid_for(n * n, 256), 256, 0, s>>>(src, n, zero_diag, complement, (float *)dst, err);
    return cudaGetLastError();
}

cudaError_t launch_pairs(int kind, const double *data, int r, int64_t n, bool fp64, int zero_diag, void *dst,
                         int *err, cudaStream_t s) {
    if (r < 1 || (kind != USTAT_LOWRANK && kind != USTAT_DIST && kind != USTAT_GRAM)) return cudaErrorInvalidValue;
    const int mode = kind == USTAT_LOWRANK ? PAIRS_LOWRANK : (kind == USTAT_GRAM ? PAIRS_GRAM : PAIRS_DIST);
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
    if (fp64) pairs_kernel<double><<<grid, block, 0, s>>>(mode, data, r, n, zero_diag, (double *)dst, err);
    else pairs_kernel<float><<<grid, block, 0, s>>>(mode, data, r, n, zero_diag, (float *)dst, err);
    return cudaGetLastError();
}

cudaError_t launch_unary_tanh(const void *X, int x_dtype, int64_t n, int d, const double *w, double *out, int *err,
                              cudaStream_t s) {
    unary_tanh_kernel<<<grid_for(n, 128), 128, 0, s>>>(X, x_dtype, n, d, w, out, err);
    return cudaGetLastError();
}

cudaError_t launch_copyvec(const double *src, int64_t n, double *dst, int *err, cudaStream_t s) {
    copyvec_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, n, dst, err);
    return cudaGetLastError();
}

cudaError_t launch_diag(const void *M, bool fp64, int64_t n, double *out, cudaStream_t s) {
    if (fp64) diag_kernel<double><<<grid_for(n, 256), 256, 0, s>>>((const double *)M, n, out);
    else diag_kernel<float><<<grid_for(n, 256), 256, 0, s>>>((const float *)M, n, out);
    return cudaGetLastError();
}

cudaError_t launch_factor_diag(int kind, double param, const void *X, int x_dtype, int d, const double *Mc,
                               int64_t n, int zero_diag, double *out, cudaStream_t s) {
    factor_diag_kernel<<<grid_for(n, 256), 256, 0, s>>>(kind, 1.0 / param, X, x_dtype, d, Mc, n, zero_diag, out,
                                                         (int)param);
    return cudaGetLastError();
}

cudaError_t launch_vmul(const double *a, const double *b, int64_t n, double *out, cudaStream_t s) {
    vmul_kernel<<<grid_for(n, 256), 256, 0, s>>>(a, b, n, out);
    return cudaGetLastError();
}

cudaError_t launch_vsum(const double *u, int64_t n, double *out, cudaStream_t s) {
    int g = (int)((n + 255) / 256);
    if (g > 152) g = 152;
    vsum_kernel<<<g, 256, 0, s>>>(u, n, out);
    return cudaGetLastError();
}

cudaError_t launch_vdot(const double *u, const double *a, int64_t n, double *out, cudaStream_t s) {
    int g = (int)((n + 255) / 256);
    if (g > 152) g = 152;
    vdot_kernel<<<g, 256, 0, s>>>(u, a, n, out);
    return cudaGetLastError();
}

cudaError_t launch_combine(const CombineEntry *entries, int nparts, int m, const double *scal, const int *err,
                           int64_t n, double *U_out, double *V_out, cudaStream_t s) {
    if (nparts <= 16) return combine_cap<16>(entries, nparts, m, scal, err, n, U_out, V_out, s);
    if (nparts <= 64) return combine_cap<64>(entries, nparts, m, scal, err, n, U_out, V_out, s);
    if (nparts <= 256) return combine_cap<256>(entries, nparts, m, scal, err, n, U_out, V_out, s);
    if (nparts <= kCombineMaxParts) return combine_cap<kCombineMaxParts>(entries, nparts, m, scal, err, n, U_out, V_out, s);
    return cudaErrorInvalidValue;
}

}  // namespace ustat
