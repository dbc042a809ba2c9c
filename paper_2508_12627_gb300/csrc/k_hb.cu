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

#include <atomic>

#include <algorithm>

#include "kcommon.cuh"
#include "kernels.h"
#include "kmath.cuh"

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

// The float32 form of the same pass for n a multiple of 4, the distinct matrices'
// count kNM fixed at compile time: each warp loads kR = 4 / kNM rows (of every
// matrix) before using them, so that every warp keeps about the same number of
// bytes in flight whatever the matrix count, and no float64 operation remains in
// the row loop (float64 is a small fraction of this part's float32 rate):
//   * a(i) becomes float32 by integer operations (d2f_rn);
//   * a reduction's row piece (eight entries times b(j), summed in float32)
//     times a(i) is added to a compensated float32 pair (TwoSum), converted to
//     float64 once at the end.
template <int kNM>
__global__ void __launch_bounds__(256, kNM <= 2 ? 2 : 3) mhbp_kernel(MhbArgs g) {
    constexpr int CB = 256;
    constexpr int kR = kNM == 1 ? 4 : (kNM == 2 ? 2 : 1);
    __shared__ __align__(16) float bsm[kMhbOps][CB];
    __shared__ float colred[8][CB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = g.n;
    const int64_t j0 = (int64_t)blockIdx.x * CB;
    auto col = [&](int c) -> int { return 4 * lane + 128 * (c >> 2) + (c & 3); };   // c < 8
    for (int o = 0; o < g.nops; ++o)
        for (int c = threadIdx.x; c < CB; c += 256) {
            const int64_t j = j0 + c;
            const double *bv = g.op[o].kind == TILE_FREDUCE ? g.op[o].b : nullptr;
            bsm[o][c] = j < n ? (bv ? d2f_rn(bv[j]) : 1.f) : 0.f;
        }
    __syncthreads();
    float fs[kMhbOps], fe[kMhbOps];
    float gacc[kMhbGemv][8];
#pragma unroll
    for (int o = 0; o < kMhbOps; ++o) fs[o] = fe[o] = 0.f;
#pragma unroll
    for (int q = 0; q < kMhbGemv; ++q)
#pragma unroll
        for (int c = 0; c < 8; ++c) gacc[q][c] = 0.f;
    const int64_t step = (int64_t)gridDim.y * 8;
    for (int64_t i = (int64_t)blockIdx.y * 8 + warp; i < n; i += kR * step) {
        float vals[kR][kNM][8];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int64_t ir = i + r * step;
#pragma unroll
            for (int m = 0; m < kNM; ++m) {
                const float *row = (const float *)g.M[m] + ir * n;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int64_t j = j0 + 4 * lane + 128 * q;   // n % 4 == 0: the piece is whole or outside
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ir < n && j < n) v = *reinterpret_cast<const float4 *>(row + j);
                    vals[r][m][4 * q + 0] = v.x;
                    vals[r][m][4 * q + 1] = v.y;
                    vals[r][m][4 * q + 2] = v.z;
                    vals[r][m][4 * q + 3] = v.w;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int64_t ir = i + r * step;
            if (ir >= n) break;
            int gi = 0;
#pragma unroll
            for (int o = 0; o < kMhbOps; ++o) {
                if (o >= g.nops) break;
                const float ai = g.op[o].a ? d2f_rn(g.op[o].a[ir]) : 1.f;
                float p[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) p[c] = 1.f;
#pragma unroll
                for (int m = 0; m < kNM; ++m) {
                    const int e = g.op[o].ex[m];
                    for (int rr = 0; rr < e; ++rr)
#pragma unroll
                        for (int c = 0; c < 8; ++c) p[c] *= vals[r][m][c];
                }
                if (g.op[o].kind == TILE_FREDUCE) {
                    const float4 b0 = *reinterpret_cast<const float4 *>(&bsm[o][4 * lane]);
                    const float4 b1 = *reinterpret_cast<const float4 *>(&bsm[o][4 * lane + 128]);
                    float sv = p[0] * b0.x;
                    sv = fmaf(p[1], b0.y, sv);
                    sv = fmaf(p[2], b0.z, sv);
                    sv = fmaf(p[3], b0.w, sv);
                    sv = fmaf(p[4], b1.x, sv);
                    sv = fmaf(p[5], b1.y, sv);
                    sv = fmaf(p[6], b1.z, sv);
                    sv = fmaf(p[7], b1.w, sv);
                    float t1, t2;
                    two_sum(fs[o], sv * ai, t1, t2);
                    fs[o] = t1;
                    fe[o] += t2;
                } else {
#pragma unroll
                    for (int q = 0; q < kMhbGemv; ++q)
                        if (q == gi) {
#pragma unroll
                            for (int c = 0; c < 8; ++c) gacc[q][c] = fmaf(ai, p[c], gacc[q][c]);
                        }
                    ++gi;
                }
            }
        }
    }
#pragma unroll
    for (int o = 0; o < kMhbOps; ++o) {
        if (o >= g.nops) break;
        if (g.op[o].kind != TILE_FREDUCE) continue;
        const double sd = block_sum((double)fs[o] + (double)fe[o]);
        if (threadIdx.x == 0) atomicAdd(g.op[o].out, sd);
    }
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
            double sd = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) sd += (double)colred[w][c];
            atomicAdd(g.op[o].out + j, sd);
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
        // grouped raster: groups of 8 tile rows, column by column inside a group
        const int64_t grp = tile / (8 * NT), rem = tile % (8 * NT);
        const int64_t gr = NT - 8 * grp < 8 ? NT - 8 * grp : 8;
        const int64_t i0 = (8 * grp + rem % gr) * kFT, j0 = (rem / gr) * kFT;
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
#pragma unroll
        for (int p = 0; p < 4; ++p) {   // unrolled: the argument arrays stay in registers
            if (p >= g.np) break;
            const T *M = (const T *)g.P[p];
            const int ex = g.pe[p];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                T x[4];
                load4(M, i0 + rr + 16 * k, j0 + cc, x);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    T f = x[e];
                    for (int q = 1; q < ex; ++q) f *= x[e];
                    v[k][e] *= f;
                }
            }
        }
        // the mirror tiles of the transposed terms into shared memory
        __syncthreads();   // the previous tile's reads are done
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (q >= g.nq) break;
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
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (q >= g.nq) break;
                    const T y = sq[q][cc + e][rr + 16 * k];   // M_q[j][i]
                    const int ex = g.qe[q];
                    for (int r = 0; r < ex; ++r) f *= y;
                }
                row = fma(f, bj[e], row);
            }
            acc = fma((double)row, g.a ? g.a[i] : 1.0, acc);
        }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) atomicAdd(g.out, s);
}

// The same reduction as a streaming pipeline, for n a multiple of the 16-byte
// piece (4 floats or 2 doubles) and 16-byte aligned matrices: every term's tile
// of the next kS - 1 tiles is in flight (cp.async, zero-filled beyond n) while
// the current one is reduced, so that the kernel keeps enough bytes in flight to
// stream at the HBM rate.  Tile: kTI rows i x 64 columns j (64 x 64 floats, 32 x
// 64 doubles: 16 KB per term).  An untransposed term's tile is kept as read
// (rows i); a transposed term's tile is its mirror (rows j, columns i) with the
// 16-byte pieces of row j permuted by j mod 8, so that 8 consecutive threads
// (consecutive j) reading the same piece index hit distinct banks.  Thread
// (jl, ig) forms the entries (i, j0 + jl) of its kTI / 4 rows: the products of
// one 16-byte piece of rows (4 or 2) times a(i) are summed in the storage type,
// then added in float64 times b(j).
__device__ __forceinline__ void cpa16(void *dst, const void *src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cpa8(void *dst, const void *src, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T>
struct FredPipe {
    static constexpr int kE = 16 / (int)sizeof(T);        // elements per 16-byte piece
    static constexpr int kTI = sizeof(T) == 4 ? 64 : 32;   // tile rows (i)
    static constexpr int kTJ = 64;                         // tile columns (j)
    static constexpr int kMat = kTI * kTJ * (int)sizeof(T);
    static constexpr int kVecBytes = 2 * 64 * 8;           // a(i), b(j) as float64
    static int stage_bytes(int nm) { return nm * kMat + kVecBytes; }
};

// kUnit: one untransposed and one transposed term, each to the first power (the
// common case; no exponent loops)
template <typename T, int kS, bool kUnit>
__global__ void __launch_bounds__(256) fredp_kernel(FredArgs g) {
    using C = FredPipe<T>;
    constexpr int kE = C::kE, kTI = C::kTI, kTJ = C::kTJ;
    constexpr bool kF = sizeof(T) == 4;
    extern __shared__ __align__(128) unsigned char fp_smem[];
    __shared__ __align__(16) float af[64];   // a(i) of the current tile in float32
    const int t = threadIdx.x;
    const int np = kUnit ? 1 : g.np, nq = kUnit ? 1 : g.nq, nm = np + nq;
    const int stage = nm * C::kMat + C::kVecBytes;
    const int n = (int)g.n;
    const int NTI = (n + kTI - 1) / kTI, NTJ = (n + kTJ - 1) / kTJ, tiles = NTI * NTJ;
    const int G = gridDim.x;
    // this thread's pieces: untransposed tiles (kTJ / kE pieces per row), mirror tiles (16 per row)
    constexpr int kPR = kTJ / kE, kPS = 256 / kPR;   // pieces per row, row step between a thread's pieces
    const int pr0 = t / kPR, pc = t % kPR;
    const int qr0 = t >> 4, qc = t & 15;

    auto coords = [&](int tile, int &i0, int &j0) {
        // grouped raster: groups of 8 tile rows, column by column inside a group, so
        // that the tiles in flight read runs of at least 8 x 256 bytes of both the
        // untransposed rows and the transposed terms' rows (DRAM page locality)
        const int grp = tile / (8 * NTJ), rem = tile - grp * 8 * NTJ;
        const int gr = NTI - 8 * grp < 8 ? NTI - 8 * grp : 8;
        const int r = gr == 8 ? (rem & 7) : rem % gr, c = gr == 8 ? (rem >> 3) : rem / gr;
        i0 = (8 * grp + r) * kTI;
        j0 = c * kTJ;
    };
    auto issue = [&](int tile, int st) {
        unsigned char *base = fp_smem + (size_t)st * stage;
        int i0, j0;
        coords(tile, i0, j0);
#pragma unroll
        for (int p = 0; p < (kUnit ? 1 : 4); ++p) {
            if (p >= np) break;
            const T *M = (const T *)g.P[p];
            const int gj = j0 + pc * kE;
            const T *src = M + (int64_t)(i0 + pr0) * n + gj;
            T *dst = (T *)(base + p * C::kMat) + pr0 * kTJ + pc * kE;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const bool ok = gj < n && i0 + pr0 + m * kPS < n;
                cpa16(dst + m * kPS * kTJ, ok ? src + (int64_t)m * kPS * n : M, ok ? 16 : 0);
            }
        }
#pragma unroll
        for (int q = 0; q < (kUnit ? 1 : 2); ++q) {
            if (q >= nq) break;
            const T *M = (const T *)g.Q[q];
            const int gi = i0 + qc * kE;
            const T *src = M + (int64_t)(j0 + qr0) * n + gi;
            T *dst = (T *)(base + (np + q) * C::kMat);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int r = qr0 + 16 * m;
                const bool ok = gi < n && j0 + r < n;
                cpa16(dst + r * kTI + (qc ^ (r & 7)) * kE, ok ? src + (int64_t)16 * m * n : M, ok ? 16 : 0);
            }
        }
        double *av = (double *)(base + nm * C::kMat), *bv = av + 64;
        if (t < kTI) {
            const int gi = i0 + t;
            if (g.a) cpa8(av + t, gi < n ? g.a + gi : g.a, gi < n ? 8 : 0);
            else av[t] = gi < n ? 1.0 : 0.0;
        } else if (t >= 64 && t < 64 + kTJ) {
            const int gj = j0 + (t - 64);
            if (g.b) cpa8(bv + (t - 64), gj < n ? g.b + gj : g.b, gj < n ? 8 : 0);
            else bv[t - 64] = gj < n ? 1.0 : 0.0;
        }
    };

    int tl = blockIdx.x;
#pragma unroll
    for (int s = 0; s < kS - 1; ++s) {
        if (tl + s * G < tiles) issue(tl + s * G, s);
        cpa_commit();
    }
    const int jl = t & 63, ig = t >> 6;
    constexpr int kPieces = kTI / 4 / kE;   // 16-byte pieces of rows per thread: 4
    double acc = 0.0;
    for (int it = 0; tl < tiles; tl += G, ++it) {
        cpa_wait<kS - 2>();
        __syncthreads();   // this tile's stage is complete; the previous stage is free
        {
            const int nt = tl + (kS - 1) * G;
            if (nt < tiles) issue(nt, (it + kS - 1) % kS);
            cpa_commit();
        }
        const unsigned char *base = fp_smem + (size_t)(it % kS) * stage;
        const T *Ps = (const T *)base;
        const T *Qs = (const T *)(base + np * C::kMat);
        const double *av = (const double *)(base + nm * C::kMat);
        if constexpr (kF) {
            // a(i) in float32 once per tile (float64 conversions are slow on this part)
            if (t < kTI) af[t] = (float)av[t];
            __syncthreads();
        }
        const double bj = av[64 + jl];
        T sum = T(0), err = T(0);   // float32: compensated (TwoSum) sum of the pieces
#pragma unroll
        for (int k = 0; k < kPieces; ++k) {
            const int c = ig * kPieces + k;   // piece index along i
            T qv[2][kE], ai[kE];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (q >= nq) break;
                const T *src = Qs + q * (kTI * kTJ) + jl * kTI + (c ^ (jl & 7)) * kE;
                if constexpr (kF) {
                    const float4 x = *reinterpret_cast<const float4 *>(src);
                    qv[q][0] = x.x, qv[q][1] = x.y, qv[q][2] = x.z, qv[q][3] = x.w;
                } else {
                    const double2 x = *reinterpret_cast<const double2 *>(src);
                    qv[q][0] = x.x, qv[q][1] = x.y;
                }
            }
            if constexpr (kF) {
                const float4 x = *reinterpret_cast<const float4 *>(&af[c * kE]);
                ai[0] = x.x, ai[1] = x.y, ai[2] = x.z, ai[3] = x.w;
            } else {
#pragma unroll
                for (int u = 0; u < kE; ++u) ai[u] = av[c * kE + u];
            }
            T grp = T(0);
#pragma unroll
            for (int u = 0; u < kE; ++u) {
                const int i = c * kE + u;
                T f;
                if constexpr (kUnit) {
                    f = Ps[i * kTJ + jl] * qv[0][u];
                } else {
                    f = T(1);
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        if (p >= np) break;
                        const T x = Ps[p * (kTI * kTJ) + i * kTJ + jl];
                        const int ex = g.pe[p];
                        for (int r = 0; r < ex; ++r) f *= x;
                    }
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        if (q >= nq) break;
                        const T y = qv[q][u];
                        const int ex = g.qe[q];
                        for (int r = 0; r < ex; ++r) f *= y;
                    }
                }
                grp = fma(f, ai[u], grp);
            }
            if constexpr (kF) {
                float s2, e2;
                two_sum(sum, grp, s2, e2);
                sum = s2;
                err += e2;
            } else {
                sum += grp;
            }
        }
        acc = fma((double)sum + (double)err, bj, acc);
    }
    cpa_wait<0>();
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
    if (!fp64 && g.n % 4 == 0) {
        // one wave: two blocks per SM (one or two matrices, more rows in flight per
        // warp) or three
        int64_t gy2 = (152 * (g.nmat <= 2 ? 2 : 3)) / gx;
        if (gy2 > maxgy) gy2 = maxgy;
        if (gy2 < 1) gy2 = 1;
        const dim3 grid2((unsigned)gx, (unsigned)gy2);
        switch (g.nmat) {
            case 1: mhbp_kernel<1><<<grid2, 256, 0, s>>>(g); break;
            case 2: mhbp_kernel<2><<<grid2, 256, 0, s>>>(g); break;
            case 3: mhbp_kernel<3><<<grid2, 256, 0, s>>>(g); break;
            default: mhbp_kernel<4><<<grid2, 256, 0, s>>>(g); break;
        }
        return cudaGetLastError();
    }
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
    static std::atomic<bool> attr[64];   // per device, set once; atomic: host threads may launch concurrently
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
    // the streaming pipeline where its 16-byte copies apply
    bool pipe = n % (fp64 ? 2 : 4) == 0 && n < (int64_t)1 << 20;   // 32-bit tile arithmetic
    for (int p = 0; p < g.np; ++p) pipe = pipe && ((uintptr_t)g.P[p] & 15) == 0;
    for (int q = 0; q < g.nq; ++q) pipe = pipe && ((uintptr_t)g.Q[q] & 15) == 0;
    if (pipe) {
        static std::atomic<bool> pattr[64];   // per device, set once; atomic: host threads may launch concurrently
        constexpr int kMaxSmem = 220 * 1024;
        if (!pattr[dev]) {
            const void *fns[] = {
                (const void *)fredp_kernel<float, 2, false>,  (const void *)fredp_kernel<float, 3, false>,
                (const void *)fredp_kernel<float, 4, false>,  (const void *)fredp_kernel<double, 2, false>,
                (const void *)fredp_kernel<double, 3, false>, (const void *)fredp_kernel<double, 4, false>,
                (const void *)fredp_kernel<float, 2, true>,   (const void *)fredp_kernel<float, 3, true>,
                (const void *)fredp_kernel<float, 4, true>,   (const void *)fredp_kernel<double, 2, true>,
                (const void *)fredp_kernel<double, 3, true>,  (const void *)fredp_kernel<double, 4, true>};
            for (const void *f : fns)
                if ((*err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem)) !=
                    cudaSuccess)
                    return true;
            pattr[dev] = true;
        }
        const int nm = g.np + g.nq;
        const int stage = fp64 ? FredPipe<double>::stage_bytes(nm) : FredPipe<float>::stage_bytes(nm);
        // two blocks per SM with the deepest ring that fits half the shared memory,
        // else one block with a ring of two or three stages
        int S = 0, bps = 2;
        for (int c = 4; c >= 2 && !S; --c)
            if (c * stage <= kMaxSmem / 2) S = c;
        if (!S) {
            bps = 1;
            S = 3 * stage <= kMaxSmem ? 3 : 2;
        }
        const int64_t ti = fp64 ? FredPipe<double>::kTI : FredPipe<float>::kTI;
        const int64_t tiles = ((n + ti - 1) / ti) * ((n + 63) / 64);
        const int grid = (int)std::min<int64_t>(tiles, 152 * bps);
        const size_t sm = (size_t)S * stage;
        const bool unit = g.np == 1 && g.nq == 1 && g.pe[0] == 1 && g.qe[0] == 1;
        if (fp64) {
            if (unit) {
                if (S == 4) fredp_kernel<double, 4, true><<<grid, 256, sm, s>>>(g);
                else if (S == 3) fredp_kernel<double, 3, true><<<grid, 256, sm, s>>>(g);
                else fredp_kernel<double, 2, true><<<grid, 256, sm, s>>>(g);
            } else {
                if (S == 4) fredp_kernel<double, 4, false><<<grid, 256, sm, s>>>(g);
                else if (S == 3) fredp_kernel<double, 3, false><<<grid, 256, sm, s>>>(g);
                else fredp_kernel<double, 2, false><<<grid, 256, sm, s>>>(g);
            }
        } else {
            if (unit) {
                if (S == 4) fredp_kernel<float, 4, true><<<grid, 256, sm, s>>>(g);
                else if (S == 3) fredp_kernel<float, 3, true><<<grid, 256, sm, s>>>(g);
                else fredp_kernel<float, 2, true><<<grid, 256, sm, s>>>(g);
            } else {
                if (S == 4) fredp_kernel<float, 4, false><<<grid, 256, sm, s>>>(g);
                else if (S == 3) fredp_kernel<float, 3, false><<<grid, 256, sm, s>>>(g);
                else fredp_kernel<float, 2, false><<<grid, 256, sm, s>>>(g);
            }
        }
        *err = cudaGetLastError();
        return true;
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
