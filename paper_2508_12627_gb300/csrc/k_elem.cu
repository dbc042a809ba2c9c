// Tensorization (the paper's Algorithm 1 for the kernel maps), vector operations
// and the final Moebius combination U = sum_pi mu_pi V_pi (Section 3.3, Lemma
// "Decomposition of U-Statistic into V-Statistics"; Algorithm 4).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kcommon.cuh"
#include "kernels.h"
#include "../../include/ustat.h"

namespace ustat {

namespace {

template <typename T>
__global__ void xconvert_kernel(const void *X, int x_dtype, int64_t total, T *out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        double v = x_dtype == 0 ? ((const double *)X)[t] : (double)((const float *)X)[t];
        out[t] = (T)v;
    }
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
__global__ void __launch_bounds__(256) kbuild_f32_kernel(int kind, float inv_param, const float *__restrict__ X,
                                                         int64_t n, int d, int zero_diag, float *__restrict__ K) {
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
            float v;
            if (kind == USTAT_RBF) {
                v = (gi == gj) ? 1.0f : exp_unbiased(-acc[r][c] * inv_param);
            } else {
                const float s = acc[r][c] + lo[r][c];
                v = s * inv_param;
            }
            if (zero_diag && gi == gj) v = 0.f;
            K[gi * n + gj] = v;
        }
    }
}

// RBF kernel matrix in float32, fused with its split into bf16 fixed-point
// slices (the row scale is known: entries lie in (0, 1], so s_j = 1).
// One block per 128 x 128 tile on or above the diagonal; the tile and its
// mirror image are written from shared memory with coalesced stores.  The
// squared distance is ||x_i||^2 + ||x_j||^2 - 2 x_i . x_j (float32; its rounding
// errors are symmetric), the exponential exp_unbiased, the diagonal exactly 1.
// slices == nullptr: K only.
constexpr int kRbfT = 128;
struct RbfArgs {
    const float *X;
    int64_t n;
    int d;
    float inv_h;
    int zero_diag;
    float *K;
    __nv_bfloat16 *slices;   // [planes][n][ldp] or null
    int64_t ldp;
    int lead_bits, planes;
    float *scales;
};

__global__ void __launch_bounds__(256) kbuild_rbf_tile_kernel(RbfArgs g) {
    extern __shared__ float sm[];
    float *xi = sm;                         // [128][33]
    float *xj = xi + kRbfT * 33;            // [128][33]
    float *S = xj + kRbfT * 33;             // [128][129]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t n = g.n;
    const int T = (int)((g.ldp + kRbfT - 1) / kRbfT);
    // upper-triangle tile t -> (tm, tn), row-major: row r starts at r T - r (r - 1) / 2
    const int t = blockIdx.x;
    const double b = 2.0 * T + 1.0;
    int tm = (int)((b - sqrt(b * b - 8.0 * t)) * 0.5);
    if (tm < 0) tm = 0;
    while (tm > 0 && tm * T - tm * (tm - 1) / 2 > t) --tm;
    while (tm + 1 < T && (tm + 1) * T - (tm + 1) * tm / 2 <= t) ++tm;
    const int tn = tm + (t - (tm * T - tm * (tm - 1) / 2));
    const int64_t i0 = (int64_t)tm * kRbfT, j0 = (int64_t)tn * kRbfT;

    // squared distances: 8 x 8 per thread (rows ty + 16 a, columns tx + 16 c)
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = 0.f;
    for (int k0 = 0; k0 < g.d; k0 += 32) {
        __syncthreads();
        for (int e = tid; e < kRbfT * 32; e += 256) {
            const int rr = e >> 5, kk = e & 31;
            const int64_t gi = i0 + rr, gj = j0 + rr;
            xi[rr * 33 + kk] = (gi < n && k0 + kk < g.d) ? g.X[gi * g.d + k0 + kk] : 0.f;
            xj[rr * 33 + kk] = (gj < n && k0 + kk < g.d) ? g.X[gj * g.d + k0 + kk] : 0.f;
        }
        __syncthreads();
        const int kmax = min(32, g.d - k0);
        for (int kk = 0; kk < kmax; ++kk) {
            float av[8], bv[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) av[a] = xi[(ty + 16 * a) * 33 + kk];
#pragma unroll
            for (int c = 0; c < 8; ++c) bv[c] = xj[(tx + 16 * c) * 33 + kk];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float df = av[a] - bv[c];
                    acc[a][c] = fmaf(df, df, acc[a][c]);
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int r = ty + 16 * a;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int cc = tx + 16 * c;
            const int64_t gi = i0 + r, gj = j0 + cc;
            float v;
            if (gi == gj) v = g.zero_diag ? 0.f : 1.f;
            else v = exp_unbiased(-acc[a][c] * g.inv_h);
            S[r * 129 + cc] = (gi < n && gj < n) ? v : 0.f;
        }
    }
    __syncthreads();
    const int64_t plane = n * g.ldp;
    const bool vec4 = (n % 4 == 0) && (g.ldp % 4 == 0);
    const float lead_scale = __int_as_float((127 + g.lead_bits) << 23);   // 2^w
    // the tile (rows i0.., cols j0..) and, off the diagonal, its mirror image;
    // each thread writes 4 consecutive columns of one row
    for (int pass = 0; pass < (tm == tn ? 1 : 2); ++pass) {
        const int64_t r0 = pass ? j0 : i0, c0 = pass ? i0 : j0;
        for (int e = tid; e < kRbfT * (kRbfT / 4); e += 256) {
            const int r = e >> 5, c = (e & 31) * 4;
            const int64_t gr = r0 + r, gc = c0 + c;
            if (gr >= n) continue;
            float v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = pass ? S[(c + q) * 129 + r] : S[r * 129 + c + q];
            if (vec4 && gc + 3 < n) {
                *reinterpret_cast<float4 *>(g.K + gr * n + gc) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (gc + q < n) g.K[gr * n + gc + q] = v[q];
            }
            if (g.slices) {
                __nv_bfloat16 dg[4][4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float y = v[q] * lead_scale;            // row scale 1: |y| <= 2^w, exact
                    float dd = rintf(y);
                    dg[0][q] = __float2bfloat16_rn(dd);
                    float sc = 1.f / 256.f;
                    for (int p = 1; p < g.planes; ++p) {
                        y = (y - dd) * 256.f;
                        dd = rintf(y);
                        dg[p][q] = __float2bfloat16_rn(dd * sc);
                        sc *= (1.f / 256.f);
                    }
                }
                __nv_bfloat16 *dst = g.slices + gr * g.ldp + gc;
                for (int p = 0; p < g.planes; ++p) {
                    if (vec4 && gc + 3 < g.ldp) {
                        uint2 w;
                        w.x = (uint32_t)__bfloat16_as_ushort(dg[p][0]) | ((uint32_t)__bfloat16_as_ushort(dg[p][1]) << 16);
                        w.y = (uint32_t)__bfloat16_as_ushort(dg[p][2]) | ((uint32_t)__bfloat16_as_ushort(dg[p][3]) << 16);
                        *reinterpret_cast<uint2 *>(dst + p * plane) = w;
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (gc + q < g.ldp) dst[p * plane + q] = dg[p][q];
                    }
                }
            }
        }
    }
    if (g.scales && tm == tn && tid < kRbfT && i0 + tid < n) g.scales[i0 + tid] = 1.f;
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

template <typename T>
__global__ void loadmat_kernel(const double *src, int64_t n, int zero_diag, T *dst) {
    const int64_t total = n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        T v = (T)src[t];
        if (zero_diag && (t / n) == (t % n)) v = 0;
        dst[t] = v;
    }
}

__global__ void unary_tanh_kernel(const void *X, int x_dtype, int64_t n, int d, const double *w, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            double x = x_dtype == 0 ? ((const double *)X)[i * d + k] : (double)((const float *)X)[i * d + k];
            s = fma(x, w[k], s);
        }
        out[i] = tanh(s);
    }
}

__global__ void copyvec_kernel(const double *src, int64_t n, double *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

template <typename T>
__global__ void diag_kernel(const T *M, int64_t n, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)M[i * n + i];
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

cudaError_t launch_xconvert(const void *X, int x_dtype, int64_t n, int d, void *Xw, bool fp64, cudaStream_t s) {
    int64_t total = n * d;
    if (fp64) xconvert_kernel<double><<<grid_for(total, 256), 256, 0, s>>>(X, x_dtype, total, (double *)Xw);
    else xconvert_kernel<float><<<grid_for(total, 256), 256, 0, s>>>(X, x_dtype, total, (float *)Xw);
    return cudaGetLastError();
}

cudaError_t launch_kbuild(int kind, double param, const void *Xw, bool fp64, int64_t n, int d, int zero_diag,
                          void *K, cudaStream_t s) {
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)((n + 63) / 64)), block(16, 16);
    if (fp64)
        kbuild_kernel<double><<<grid, block, 0, s>>>(kind, 1.0 / param, (const double *)Xw, n, d, zero_diag,
                                                     (double *)K);
    else
        kbuild_f32_kernel<<<grid, block, 0, s>>>(kind, (float)(1.0 / param), (const float *)Xw, n, d, zero_diag,
                                                 (float *)K);
    return cudaGetLastError();
}

cudaError_t launch_kbuild_rbf(const float *Xw, int64_t n, int d, double param, int zero_diag, float *K,
                              void *slices, int64_t ldp, int lead_bits, int planes, float *scales, cudaStream_t s) {
    RbfArgs g{Xw, n, d, (float)(1.0 / param), zero_diag, K, (__nv_bfloat16 *)slices, slices ? ldp : n, lead_bits,
              planes, slices ? scales : nullptr};
    const int smem = (2 * kRbfT * 33 + kRbfT * 129) * 4;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kbuild_rbf_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t T = (g.ldp + kRbfT - 1) / kRbfT;
    kbuild_rbf_tile_kernel<<<(unsigned)(T * (T + 1) / 2), 256, smem, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_loadmat(const double *src, int64_t n, bool fp64, int zero_diag, void *dst, cudaStream_t s) {
    if (fp64) loadmat_kernel<double><<<grid_for(n * n, 256), 256, 0, s>>>(src, n, zero_diag, (double *)dst);
    else loadmat_kernel<float><<<grid_for(n * n, 256), 256, 0, s>>>(src, n, zero_diag, (float *)dst);
    return cudaGetLastError();
}

cudaError_t launch_unary_tanh(const void *X, int x_dtype, int64_t n, int d, const double *w, double *out,
                              cudaStream_t s) {
    unary_tanh_kernel<<<grid_for(n, 128), 128, 0, s>>>(X, x_dtype, n, d, w, out);
    return cudaGetLastError();
}

cudaError_t launch_copyvec(const double *src, int64_t n, double *dst, cudaStream_t s) {
    copyvec_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_diag(const void *M, bool fp64, int64_t n, double *out, cudaStream_t s) {
    if (fp64) diag_kernel<double><<<grid_for(n, 256), 256, 0, s>>>((const double *)M, n, out);
    else diag_kernel<float><<<grid_for(n, 256), 256, 0, s>>>((const float *)M, n, out);
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

cudaError_t launch_combine(const CombineEntry *entries, int nparts, int m, const double *scal, const int *err,
                           int64_t n, double *U_out, double *V_out, cudaStream_t s) {
    if (nparts <= 16) return combine_cap<16>(entries, nparts, m, scal, err, n, U_out, V_out, s);
    if (nparts <= 64) return combine_cap<64>(entries, nparts, m, scal, err, n, U_out, V_out, s);
    if (nparts <= 256) return combine_cap<256>(entries, nparts, m, scal, err, n, U_out, V_out, s);
    if (nparts <= kCombineMaxParts) return combine_cap<kCombineMaxParts>(entries, nparts, m, scal, err, n, U_out, V_out, s);
    return cudaErrorInvalidValue;
}

}  // namespace ustat
