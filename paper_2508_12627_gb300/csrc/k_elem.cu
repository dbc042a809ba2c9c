// Tensorization (the paper's Algorithm 1 for the kernel maps), vector operations
// and the final Moebius combination U = sum_pi mu_pi V_pi (Section 3.3, Lemma
// "Decomposition of U-Statistic into V-Statistics"; Algorithm 4).
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
// U_mean = U_sum / (n)_m.  One thread: at most 877 terms.
__global__ void combine_kernel(const CombineTable tab, const double *scal, const int *err, int64_t n,
                               double *U_out, double *V_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const bool bad = err && *err != 0;
    Neumaier acc;
    const double dn = (double)n;
    for (int p = 0; p < tab.nparts; ++p) {
        double v = 0.0;
        if (tab.evaluated[p]) {
            v = 1.0;
            for (int q = 0; q < kCombineMaxScal; ++q) {
                unsigned short s = tab.sid[p][q];
                if (s != 0xffff) v *= scal[s];
            }
            for (int q = 0; q < tab.nfree[p]; ++q) v *= dn;
        }
        if (bad) v = nan("");
        if (V_out) V_out[p] = v;
        acc.add((double)tab.mu[p] * v);
    }
    double ff = 1.0;
    for (int q = 0; q < tab.m; ++q) ff *= (dn - q);
    const double u = bad ? nan("") : acc.value();
    U_out[0] = u;
    U_out[1] = u / ff;
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

cudaError_t launch_combine(const CombineTable &tab, const double *scal, const int *err, int64_t n, double *U_out,
                           double *V_out, cudaStream_t s) {
    combine_kernel<<<1, 32, 0, s>>>(tab, scal, err, n, U_out, V_out);
    return cudaGetLastError();
}

}  // namespace ustat
