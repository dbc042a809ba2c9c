// The s = 2 and s = 3 elimination steps (Appendix D: summing out an index with
// two or three live neighbours) on CUDA cores, in float32 or float64:
//
//   C(j, k)  = sum_i A(i, j) u(i) B(i, k)                          (stored and/or)
//   out_r   += sum_jk C(j, k)^p_r W_r(j, k) a_r(j) b_r(k)          (fused reductions)
//   GEMM3   : for every bb, the same with u'(i) = u(i) Ab(i, bb) and the
//             extra epilogue weights Wbc(bb, j), Wbd(bb, k), ub(bb)  (grid.z = bb)
//
// Register-blocked tiles (BM x BN, TM x TN per thread, 16 x 16 threads).
// Reductions accumulate in float64 and add one value per block and reduction.
// With `symmetric` only tiles on or above the diagonal run and off-diagonal
// tiles count twice.
#include <cuda_runtime.h>

#include "kcommon.cuh"
#include "kernels.h"

namespace ustat {

namespace {

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(256) simt_gemm_kernel(SimtGemmArgs g) {
    static_assert(BM == BN, "square tiles");
    __shared__ T As[BK][BM];
    __shared__ T Bs[BK][BN];
    __shared__ T rw[BM];   // epilogue row weights
    __shared__ T cw[BN];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 16 + tx;
    const int64_t n = g.n;
    if (g.symmetric && blockIdx.y > blockIdx.x) return;
    const int64_t j0 = (int64_t)blockIdx.y * BM, k0 = (int64_t)blockIdx.x * BN;
    const int64_t bb = blockIdx.z;
    const T *A = (const T *)g.A;
    const T *B = (const T *)g.B;
    const T *Ab = (const T *)g.Ab;
    T acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = 0;

    for (int64_t i0 = 0; i0 < n; i0 += BK) {
        // A tile (i, j), scaled by u(i) [and Ab(i, bb)]
        for (int e = tid; e < BK * BM; e += 256) {
            int kk, jj;
            if (g.transA) { jj = e / BK; kk = e % BK; }
            else { kk = e / BM; jj = e % BM; }
            int64_t i = i0 + kk, j = j0 + jj;
            T v = 0;
            if (i < n && j < n) {
                v = g.transA ? A[j * n + i] : A[i * n + j];
                if (g.u) v *= (T)g.u[i];
                if (g.gemm3) v *= g.transAb ? Ab[bb * n + i] : Ab[i * n + bb];
            }
            As[kk][jj] = v;
        }
        for (int e = tid; e < BK * BN; e += 256) {
            int kk, cc;
            if (g.transB) { cc = e / BK; kk = e % BK; }
            else { kk = e / BN; cc = e % BN; }
            int64_t i = i0 + kk, k = k0 + cc;
            T v = 0;
            if (i < n && k < n) v = g.transB ? B[k * n + i] : B[i * n + k];
            Bs[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[TM], bv[TN];
#pragma unroll
            for (int r = 0; r < TM; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < TN; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
        }
        __syncthreads();
    }

    if (g.C) {
        T *C = (T *)g.C;
#pragma unroll
        for (int r = 0; r < TM; ++r) {
            int64_t j = j0 + ty + 16 * r;
            if (j >= n) continue;
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                int64_t k = k0 + tx + 16 * c;
                if (k < n) C[j * n + k] = acc[r][c];
            }
        }
    }
    const double wgt = (g.symmetric && blockIdx.x != blockIdx.y) ? 2.0 : 1.0;
    for (int q = 0; q < g.nred; ++q) {
        const SimtRed &R = g.red[q];
        const T *W = (const T *)R.W;
        const T *Wbc = (const T *)g.Wbc;
        const T *Wbd = (const T *)g.Wbd;
        __syncthreads();
        for (int e = tid; e < BM; e += 256) {
            int64_t j = j0 + e;
            T v = 0;
            if (j < n) {
                v = R.a ? (T)R.a[j] : T(1);
                if (g.gemm3 && Wbc) v *= g.transWbc ? Wbc[j * n + bb] : Wbc[bb * n + j];
            }
            rw[e] = v;
        }
        for (int e = tid; e < BN; e += 256) {
            int64_t k = k0 + e;
            T v = 0;
            if (k < n) {
                v = R.b ? (T)R.b[k] : T(1);
                if (g.gemm3 && Wbd) v *= g.transWbd ? Wbd[k * n + bb] : Wbd[bb * n + k];
            }
            cw[e] = v;
        }
        __syncthreads();
        double s = 0.0;
#pragma unroll
        for (int r = 0; r < TM; ++r) {
            int64_t j = j0 + ty + 16 * r;
            if (j >= n) continue;
            T rowp = 0;
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                int64_t k = k0 + tx + 16 * c;
                if (k >= n) continue;
                T w = cw[tx + 16 * c];
                if (W) w *= R.transW ? W[k * n + j] : W[j * n + k];
                const T x = R.pow == 2 ? acc[r][c] * acc[r][c] : acc[r][c];
                rowp = fma(x, w, rowp);
            }
            s += (double)rowp * (double)rw[ty + 16 * r];
        }
        if (g.gemm3 && g.ub) s *= g.ub[bb];
        s = block_sum(s * wgt);
        if (tid == 0) atomicAdd(R.out, s);
    }
}

}  // namespace

cudaError_t launch_gemm_simt(const SimtGemmArgs &g0, bool fp64, cudaStream_t s) {
    SimtGemmArgs g = g0;
    if (g.C || g.gemm3) g.symmetric = 0;
    if (g.nred < 0 || g.nred > 4) return cudaErrorInvalidValue;
    const int64_t n = g.n;
    const unsigned zb = g.gemm3 ? (unsigned)n : 1u;
    dim3 block(16, 16);
    if (fp64) {
        dim3 grid((unsigned)((n + 63) / 64), (unsigned)((n + 63) / 64), zb);
        simt_gemm_kernel<double, 64, 64, 8, 4, 4><<<grid, block, 0, s>>>(g);
    } else {
        dim3 grid((unsigned)((n + 127) / 128), (unsigned)((n + 127) / 128), zb);
        simt_gemm_kernel<float, 128, 128, 8, 8, 8><<<grid, block, 0, s>>>(g);
    }
    return cudaGetLastError();
}

}  // namespace ustat
