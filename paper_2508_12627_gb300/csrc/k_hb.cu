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

#include <algorithm>

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

// Several reductions / GEMVs over the same (untransposed) matrices in one pass:
// each block owns 512 columns and a slice of the rows; every warp reads whole
// 512-column row segments (float4 when the row length allows it) of each
// distinct matrix once and evaluates every operation on them.  Operation o
// multiplies matrix m ex[o][m] times (the terms of a merged factor).
// GEMV partial sums accumulate in the matrices' own type (float64 for float64
// storage, whose point is to keep every rounding below float32's).
template <typename T, bool kVec>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : 3) mhb_kernel(MhbArgs g) {
    constexpr int CB = 256;   // columns per block: 8 per lane
    __shared__ T bsm[kMhbOps][CB];
    __shared__ T colred[8][CB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = g.n;
    const int64_t j0 = (int64_t)blockIdx.x * CB;
    auto col = [&](int c) -> int { return kVec ? (4 * lane + 128 * (c >> 2) + (c & 3)) : (lane + 32 * c); };  // c < 8
    for (int o = 0; o < g.nops; ++o)
        for (int c = threadIdx.x; c < CB; c += 256) {
            const int64_t j = j0 + c;
            const double *bv = g.op[o].kind == TILE_FREDUCE ? g.op[o].b : nullptr;
            bsm[o][c] = j < n ? (bv ? (T)bv[j] : T(1)) : T(0);
        }
    __syncthreads();
    double facc[kMhbOps];
    T gacc[kMhbGemv][8];
#pragma unroll
    for (int o = 0; o < kMhbOps; ++o) facc[o] = 0.0;
#pragma unroll
    for (int q = 0; q < kMhbGemv; ++q)
#pragma unroll
        for (int c = 0; c < 8; ++c) gacc[q][c] = T(0);
    for (int64_t i = (int64_t)blockIdx.y * 8 + warp; i < n; i += (int64_t)gridDim.y * 8) {
        T vals[kMhbMats][8];
#pragma unroll
        for (int m = 0; m < kMhbMats; ++m) {
            if (m >= g.nmat) break;
            const T *row = (const T *)g.M[m] + i * n;
            if constexpr (kVec) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int64_t j = j0 + 4 * lane + 128 * q;
                    if (j + 3 < n) {
                        const float4 v = *reinterpret_cast<const float4 *>(row + j);
                        vals[m][4 * q + 0] = v.x;
                        vals[m][4 * q + 1] = v.y;
                        vals[m][4 * q + 2] = v.z;
                        vals[m][4 * q + 3] = v.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) vals[m][4 * q + e] = (j + e < n) ? row[j + e] : T(0);
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int64_t j = j0 + col(c);
                    vals[m][c] = j < n ? row[j] : T(0);
                }
            }
        }
        int gi = 0;
#pragma unroll
        for (int o = 0; o < kMhbOps; ++o) {
            if (o >= g.nops) break;
            const double ai = g.op[o].a ? g.op[o].a[i] : 1.0;
            T p[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) p[c] = T(1);
#pragma unroll
            for (int m = 0; m < kMhbMats; ++m) {
                const int e = g.op[o].ex[m];
                for (int r = 0; r < e; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) p[c] *= vals[m][c];
            }
            if (g.op[o].kind == TILE_FREDUCE) {
                T s = 0;
#pragma unroll
                for (int c = 0; c < 8; ++c) s = fma(p[c], bsm[o][col(c)], s);
                facc[o] += (double)s * ai;
            } else {
                const T af = (T)ai;
#pragma unroll
                for (int q = 0; q < kMhbGemv; ++q)
                    if (q == gi) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) gacc[q][c] = fma(af, p[c], gacc[q][c]);
                    }
                ++gi;
            }
        }
    }
    // FREDUCE: block sums
#pragma unroll
    for (int o = 0; o < kMhbOps; ++o) {
        if (o >= g.nops) break;
        if (g.op[o].kind != TILE_FREDUCE) continue;
        const double s = block_sum(facc[o]);
        if (threadIdx.x == 0) atomicAdd(g.op[o].out, s);
    }
    // GEMV: column sums across the 8 warps
    int gi = 0;
    for (int o = 0; o < g.nops; ++o) {
        if (g.op[o].kind != TILE_GEMV) continue;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kMhbGemv; ++q)
            if (q == gi) {
#pragma unroll
                for (int c = 0; c < 8; ++c) colred[warp][col(c)] = gacc[q][c];
            }
        __syncthreads();
        for (int c = threadIdx.x; c < CB; c += 256) {
            const int64_t j = j0 + c;
            if (j >= n) continue;
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) s += (double)colred[w][c];
            atomicAdd(g.op[o].out + j, s);
        }
        ++gi;
    }
}

// The terminal reduction sum_ij prod_t term_t(i, j) a(i) b(j) with transposed
// terms, on 64 x 64 tiles: the distinct untransposed matrices are read by each
// thread straight from global memory (16-byte loads along rows), the distinct
// transposed ones (term M^T: M[j][i]) are read the same way as their mirror tile
// (rows J, columns I) into shared memory, and each thread forms its 16 entries
// (four rows, four consecutive columns) with every term raised to its
// multiplicity.  Each row's four products times b(j) are summed in the storage
// type and then added in float64 times a(i): one float64 operation per four
// entries (this part's float64 pipe is a small fraction of its float32 rate).
struct FredArgs {
    const void *P[4];   // untransposed distinct matrices
    int pe[4];          // their multiplicities
    int np;
    const void *Q[2];   // transposed distinct matrices
    int qe[2];
    int nq;
    int64_t n;
    const double *a, *b;
    double *out;
};

constexpr int kFT = 64;   // tile edge

template <typename T, bool kVec>
__global__ void __launch_bounds__(256) fred_kernel(FredArgs g) {
    extern __shared__ __align__(16) unsigned char fred_smem[];
    T(*sq)[kFT][kFT + 1] = reinterpret_cast<T(*)[kFT][kFT + 1]>(fred_smem);
    const int t = threadIdx.x;
    const int rr = t >> 4;          // rows rr + 16 k of the tile
    const int cc = (t & 15) * 4;    // columns cc .. cc + 3
    const int64_t n = g.n;
    const int64_t NT = (n + kFT - 1) / kFT;
    double acc = 0.0;
    for (int64_t tile = blockIdx.x; tile < NT * NT; tile += gridDim.x) {
        const int64_t i0 = (tile / NT) * kFT, j0 = (tile % NT) * kFT;
        // four consecutive entries of row `row`, from column `col` on (zero outside)
        auto load4 = [&](const T *M, int64_t row, int64_t col, T (&v)[4]) {
            if (row < n && kVec && col + 3 < n) {
                if constexpr (sizeof(T) == 4) {
                    const float4 x = *reinterpret_cast<const float4 *>(M + row * n + col);
                    v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
                } else {
                    const double2 x0 = *reinterpret_cast<const double2 *>(M + row * n + col);
                    const double2 x1 = *reinterpret_cast<const double2 *>(M + row * n + col + 2);
                    v[0] = x0.x, v[1] = x0.y, v[2] = x1.x, v[3] = x1.y;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = (row < n && col + e < n) ? M[row * n + col + e] : T(0);
            }
        };
        // the product of the untransposed terms, straight from global memory
        T v[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e) v[k][e] = T(1);
        for (int p = 0; p < g.np; ++p) {
            const T *M = (const T *)g.P[p];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                T x[4];
                load4(M, i0 + rr + 16 * k, j0 + cc, x);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    T f = x[e];
                    for (int q = 1; q < g.pe[p]; ++q) f *= x[e];
                    v[k][e] *= f;
                }
            }
        }
        // the mirror tiles of the transposed terms into shared memory
        __syncthreads();   // the previous tile's reads are done
        for (int q = 0; q < g.nq; ++q) {
            const T *M = (const T *)g.Q[q];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                T x[4];
                load4(M, j0 + rr + 16 * k, i0 + cc, x);
#pragma unroll
                for (int e = 0; e < 4; ++e) sq[q][rr + 16 * k][cc + e] = x[e];
            }
        }
        __syncthreads();
        T bj[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int64_t j = j0 + cc + e;
            bj[e] = j < n ? (g.b ? (T)g.b[j] : T(1)) : T(0);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + rr + 16 * k;
            if (i >= n) continue;
            T row = T(0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                T f = v[k][e];
                for (int q = 0; q < g.nq; ++q) {
                    const T y = sq[q][cc + e][rr + 16 * k];   // M_q[j][i]
                    for (int r = 0; r < g.qe[q]; ++r) f *= y;
                }
                row = fma(f, bj[e], row);
            }
            acc = fma((double)row, g.a ? g.a[i] : 1.0, acc);
        }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) atomicAdd(g.out, s);
}

}  // namespace

cudaError_t launch_mhb(const MhbArgs &g0, bool fp64, cudaStream_t s) {
    MhbArgs g = g0;
    if (g.nmat < 1 || g.nmat > kMhbMats || g.nops < 1 || g.nops > kMhbOps) return cudaErrorInvalidValue;
    int ngemv = 0;
    for (int o = 0; o < g.nops; ++o) {
        for (int m = 0; m < kMhbMats; ++m) g.op[o].ex[m] = 0;
        for (int t = 0; t < g.op[o].nt; ++t) {
            const int m = g.op[o].mat[t];
            if (m < 0 || m >= g.nmat) return cudaErrorInvalidValue;
            g.op[o].ex[m]++;
        }
        if (g.op[o].kind == TILE_GEMV) ++ngemv;
    }
    if (ngemv > kMhbGemv) return cudaErrorInvalidValue;
    const int64_t gx = (g.n + 255) / 256;
    int64_t gy = (2 * 152 + gx - 1) / gx;
    const int64_t maxgy = (g.n + 7) / 8;
    if (gy > maxgy) gy = maxgy;
    if (gy < 1) gy = 1;
    dim3 grid((unsigned)gx, (unsigned)gy);
    if (fp64) mhb_kernel<double, false><<<grid, 256, 0, s>>>(g);
    else if (g.n % 4 == 0) mhb_kernel<float, true><<<grid, 256, 0, s>>>(g);
    else mhb_kernel<float, false><<<grid, 256, 0, s>>>(g);
    return cudaGetLastError();
}

namespace {

// FREDUCE with transposed terms on the 64 x 64 tile kernel: the terms grouped into
// distinct matrices with multiplicities; false where it does not apply (more than
// two distinct transposed matrices, or none)
bool launch_fred(const TileTerms &tt, bool fp64, int64_t n, const double *a, const double *b, double *out,
                 cudaStream_t s, cudaError_t *err) {
    FredArgs g{};
    for (int t = 0; t < tt.nt; ++t) {
        const bool tr = tt.trans[t] != 0;
        const void **L = tr ? g.Q : g.P;
        int *E = tr ? g.qe : g.pe;
        int &cnt = tr ? g.nq : g.np;
        int f = -1;
        for (int q = 0; q < cnt; ++q)
            if (L[q] == tt.M[t]) f = q;
        if (f < 0) {
            if (cnt == (tr ? 2 : 4)) return false;
            L[cnt] = tt.M[t];
            E[cnt] = 0;
            f = cnt++;
        }
        E[f]++;
    }
    if (g.nq == 0) return false;
    g.n = n;
    g.a = a;
    g.b = b;
    g.out = out;
    const size_t smem = (size_t)g.nq * kFT * (kFT + 1) * (fp64 ? 8 : 4);
    static bool attr[64] = {false};
    int dev = 0;
    if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return true;
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return true;
    }
    if (!attr[dev]) {
        const int big = 2 * kFT * (kFT + 1) * 8;
        const void *fns[] = {(const void *)fred_kernel<float, true>, (const void *)fred_kernel<float, false>,
                             (const void *)fred_kernel<double, true>, (const void *)fred_kernel<double, false>};
        for (const void *f : fns)
            if ((*err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess)
                return true;
        attr[dev] = true;
    }
    const int64_t NT = (n + kFT - 1) / kFT;
    const int64_t tiles = NT * NT;
    const int grid = (int)std::min<int64_t>(tiles, 152 * 6);
    const bool vec = n % 4 == 0;
    if (fp64) {
        if (vec) fred_kernel<double, true><<<grid, 256, smem, s>>>(g);
        else fred_kernel<double, false><<<grid, 256, smem, s>>>(g);
    } else {
        if (vec) fred_kernel<float, true><<<grid, 256, smem, s>>>(g);
        else fred_kernel<float, false><<<grid, 256, smem, s>>>(g);
    }
    *err = cudaGetLastError();
    return true;
}

}  // namespace

cudaError_t launch_tile_op(int mode, const TileTerms &tt, bool fp64, int64_t n, const double *a, const double *b,
                           void *out, cudaStream_t s) {
    if (mode == TILE_FREDUCE) {
        cudaError_t e = cudaSuccess;
        if (launch_fred(tt, fp64, n, a, b, (double *)out, s, &e)) return e;
    }
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
