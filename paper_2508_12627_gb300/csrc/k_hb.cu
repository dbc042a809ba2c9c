// HBM-bound operations over up to four oriented n x n factor terms: Hadamard
// merge of parallel factors, the s = 1 elimination step (a weighted column sum,
// i.e. a GEMV, Appendix D with one live neighbour) and the terminal reduction
// sum_ij prod_t F_t(i, j) a(i) b(j) that ends a component (s = 1 steps and
// Frobenius-type reductions against a stored product).
//
// Tiling: a block covers 32 columns and walks row tiles of 32 (grid-stride in
// rows); 32 x 8 threads, 4 rows per thread.  A transposed term is staged through
// shared memory so that every global read is a 128-byte row segment.
#include <cuda_runtime.h>

#include "kcommon.cuh"
#include "kernels.h"

namespace ustat {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) tile_kernel(int mode, TileTerms tt, int64_t n, const double *__restrict__ a,
                                                   const double *__restrict__ b, void *out) {
    __shared__ T stile[4][32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    const int64_t j = j0 + tx;
    const bool jok = j < n;
    const double bj = (b && jok) ? b[j] : 1.0;
    double red = 0.0;      // FREDUCE partial
    double colsum = 0.0;   // GEMV partial for column j
    const int64_t ntile = (n + 31) / 32;
    bool any_trans = false;
    for (int t = 0; t < tt.nt; ++t) any_trans |= tt.trans[t] != 0;
    for (int64_t it = blockIdx.y; it < ntile; it += gridDim.y) {
        const int64_t i0 = it * 32;
        if (any_trans) {
            __syncthreads();
            for (int t = 0; t < tt.nt; ++t) {
                if (!tt.trans[t]) continue;
                const T *M = (const T *)tt.M[t];
                // stile[t][jj][ii] = M[j0 + jj][i0 + ii] (coalesced along ii)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    int jj = ty + 8 * r;
                    int64_t gj = j0 + jj, gi = i0 + tx;
                    stile[t][jj][tx] = (gj < n && gi < n) ? M[gj * n + gi] : T(0);
                }
            }
            __syncthreads();
        }
        T part = 0;
        double dpart = 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int ii = ty + 8 * r;
            const int64_t i = i0 + ii;
            if (i >= n || !jok) continue;
            T v = 1;
            for (int t = 0; t < tt.nt; ++t) {
                T x = tt.trans[t] ? stile[t][tx][ii] : ((const T *)tt.M[t])[i * n + j];
                v *= x;
            }
            if (mode == TILE_HADAMARD) {
                ((T *)out)[i * n + j] = v;
            } else if (mode == TILE_GEMV) {
                if (a) dpart += a[i] * (double)v;
                else part += v;
            } else {
                double w = (double)v;
                if (a) w *= a[i];
                dpart += w;
            }
        }
        if (mode == TILE_GEMV) colsum += dpart + (double)part;
        else if (mode == TILE_FREDUCE) red += dpart;
    }
    if (mode == TILE_GEMV) {
        __shared__ double cs[8][32];
        cs[ty][tx] = colsum;
        __syncthreads();
        if (ty == 0 && jok) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) s += cs[q][tx];
            atomicAdd((double *)out + j, s);
        }
    } else if (mode == TILE_FREDUCE) {
        double s = block_sum(red * bj);
        if (tx == 0 && ty == 0) atomicAdd((double *)out, s);
    }
}

}  // namespace

cudaError_t launch_tile_op(int mode, const TileTerms &tt, bool fp64, int64_t n, const double *a, const double *b,
                           void *out, cudaStream_t s) {
    const int64_t nt = (n + 31) / 32;
    int64_t gy = (152 * 8 + nt - 1) / nt;
    if (mode == TILE_HADAMARD) gy = nt;
    if (gy > nt) gy = nt;
    if (gy < 1) gy = 1;
    dim3 grid((unsigned)nt, (unsigned)gy), block(32, 8);
    if (fp64) tile_kernel<double><<<grid, block, 0, s>>>(mode, tt, n, a, b, out);
    else tile_kernel<float><<<grid, block, 0, s>>>(mode, tt, n, a, b, out);
    return cudaGetLastError();
}

}  // namespace ustat
