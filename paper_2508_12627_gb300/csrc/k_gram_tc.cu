// RBF kernel matrix K(i, j) = exp(-||x_i - x_j||^2 / h) built from the Gram
// matrix X X^T on the tensor cores (tcgen05 + TMA, sm_103a): the tensorization
// step of the method (Section 3.1, Algorithm 1) for a pairwise factor that
// depends on the sample only through inner products.
//
// Accuracy.  The squared distance is formed as ||x_i||^2 + ||x_j||^2 - 2 x_i.x_j:
//   * every row of X is split into four bf16 fixed-point digit planes relative to
//     a power-of-two row scale (32 bits of the row's largest coordinate);
//   * the leading digit product accumulates exactly (integers below 2^24) in its
//     own TMEM accumulator, the nine products of weight 2^-8 .. 2^-24 in a second;
//   * the squared norms are float64 sums of the given coordinates, carried as
//     float pairs;
//   * the three-term sum is formed with two TwoSum steps, so that a near pair's
//     cancellation loses nothing and every other rounding is symmetric;
//   * the diagonal is exactly 1 (0 in the sparsified mode).
// The exponential is the same unbiased float32 exp as the direct-difference
// build, so both builds give K to float32 rounding.
//
// Kernel.  Persistent CTAs, one per SM, over the tiles on or above the diagonal
// (K is symmetric).  Warp 0 streams the two operand tiles (rows of the tile's
// row block and column block) with TMA; warp 1 issues ten tcgen05.mma per
// 16-wide k step into one of two TMEM accumulator pairs; sixteen epilogue warps
// (four per TMEM lane quadrant, 32 columns each) form K, its bf16 digit planes
// (row scale 1) and up to four fused reductions of entrywise powers of K, and
// store the tile and, off the diagonal, its mirror (coalesced across lanes).
// Every mbarrier wait is bounded; an abort records the error word, drains the
// MMAs and copies in flight and frees the TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>

#include "kcommon.cuh"
#include "kernels.h"
#include "kmath.cuh"
#include "tc_ptx.cuh"

namespace ustat {

namespace {

using namespace tc;

constexpr int kGP = 4;                             // digit planes of X
constexpr int kGT = 128;                           // tile rows = tile columns
constexpr int kGRowBytes = 64;                     // one k-block: 32 bf16 per row
constexpr int kGBK = kGRowBytes / 2;
constexpr int kGEpiWarps = 16;
constexpr int kGThreads = 32 * (2 + kGEpiWarps);
constexpr int kGStages = 2;
constexpr int kGTile = kGT * kGRowBytes;           // one plane of one operand tile
constexpr int kGStageBytes = 2 * kGP * kGTile;     // both operands
constexpr int kGAccCols = 2 * kGT;                 // [hi | lo]
constexpr int kGTmemCols = 2 * kGAccCols;          // two accumulator pairs
constexpr int kGBarBytes = 256;                    // barriers and flags
// per epilogue warp: a 32 x 16 chunk of K (rows padded to 17 floats), its digits
// as 32 rows of 8 bf16 pairs (padded to 9) and transposed as 16 rows of 32 bf16
// (padded to 40, keeping 16-byte alignment)
struct EpiStage {
    float kf[32][17];
    uint32_t dr[32][9];
    alignas(16) unsigned short dt[16][40];
    float4 cd[32];   // the warp's 32 columns: scale factor and squared norm (hi, lo)
};
constexpr int kGSmem = kGStages * kGStageBytes + kGBarBytes + kGEpiWarps * (int)sizeof(EpiStage) + 1024;
constexpr int kGMaxRed = 4;
constexpr long long kGWaitLimit = 4000000000LL;

struct GramRed {
    int pow;      // 1..4
    int vec;      // 1: out[i] += sum_j K_ij^pow; 0: *out += sum_ij K_ij^pow
    double *out;
};

struct GramArgs {
    int64_t n;
    int num_k;            // k-blocks of 32 coordinates
    int lead_x;           // leading digit bits of the X digits
    const float *sx;      // [npad] row scales of the X digits (powers of two)
    const float2 *nrm;    // [npad] ||x_i||^2 as a (hi, lo) float pair
    float inv_h;
    int zero_diag;
    float *K;             // n x n float32 (row-major)
    int upper_only;       // K itself only on and above the diagonal tiles
    __nv_bfloat16 *slices;   // [planes][n][ldp] digits of K (may be null)
    int64_t ldp;
    int lead_k, planes;
    float *scales;        // [n] digit row scales of K (all 1)
    int nred;
    GramRed red[kGMaxRed];
    int *err;
    long long wait_limit;
    // window (memory-lean evaluation): the tiles of rows row0 .. row0 + rows - 1 and
    // columns col0 .. col0 + cols - 1 (multiples of 128 for row0, col0), every one
    // computed (no mirror); K may be null (not stored), and K, scales and the
    // reduction vectors keep global indices (the caller offsets the pointers of
    // buffers that hold only the window); the digit planes hold row j at
    // (j - srow0), plane stride splane elements.  Used by the kWin form only.
    int64_t row0, rows, col0, cols;
    int64_t srow0, splane;
    // work units (set by the launcher for its grid): units 0 .. nfull - 1 are whole
    // tiles, units nfull .. units - 1 the column halves of the last tiles
    int nfull, units;
};

// Row i of X: its digits (kGP planes of ldx coordinates, zero beyond d), its
// power-of-two scale and its squared norm in float64 (kept as a float pair);
// rows n .. npad - 1 get scale 1 and norm 0.  A non-finite coordinate sets the
// error word.  One warp per row.
__global__ void __launch_bounds__(256) gram_xsplit_kernel(const void *X, int x_dtype, int64_t n, int64_t npad, int d,
                                                          int ldx, int lead, __nv_bfloat16 *dig, float *sx,
                                                          float2 *nrm, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= npad) return;
    if (i >= n) {
        if (lane == 0) {
            sx[i] = 1.f;
            nrm[i] = make_float2(0.f, 0.f);
        }
        return;
    }
    auto ld = [&](int k) -> double {
        return x_dtype == 0 ? ((const double *)X)[i * d + k] : (double)((const float *)X)[i * d + k];
    };
    double mx = 0.0, s = 0.0;
    bool bad = false;
    for (int k = lane; k < d; k += 32) {
        const double v = ld(k);
        bad |= !isfinite(v);
        mx = fmax(mx, fabs(v));
        s = fma(v, v, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (bad && err) atomicOr(err, kErrWordNonfinite);
    const int e = row_exp(mx);
    if (lane == 0) {
        sx[i] = ldexpf(1.f, e);
        const float hi = (float)s;
        nrm[i] = make_float2(hi, (float)(s - (double)hi));
    }
    const int64_t plane = n * ldx;
    for (int k = lane; k < ldx; k += 32)
        write_digits(k < d && isfinite(mx) ? ld(k) : 0.0, lead, e, kGP, dig + i * ldx + k, plane);
}

// upper-triangle tile t -> (tm, tn), row-major: row r starts at r T - r (r - 1) / 2
__device__ __forceinline__ void upper_tile(int t, int T, int &tm, int &tn) {
    const double b = 2.0 * T + 1.0;
    int r = (int)((b - sqrt(b * b - 8.0 * t)) * 0.5);
    if (r < 0) r = 0;
    while (r > 0 && r * T - r * (r - 1) / 2 > t) --r;
    while (r + 1 < T && (r + 1) * T - (r + 1) * r / 2 <= t) ++r;
    tm = r;
    tn = r + (t - (r * T - r * (r - 1) / 2));
}

// x^p for p in 1..4 (p uniform across the warp)
__device__ __forceinline__ float powk(float x, int p) {
    const float x2 = x * x;
    return p == 1 ? x : (p == 2 ? x2 : (p == 3 ? x2 * x : x2 * x2));
}

// the sum over the 32 lanes of each of 16 per-lane values, by halving exchanges:
// lane l ends with column ((l >> 4) & 1) * 8 + ((l >> 3) & 1) * 4 + ((l >> 2) & 1) * 2
// + ((l >> 1) & 1), both lanes of a pair holding it
__device__ __forceinline__ float transpose_reduce16(float (&v)[16], int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool up = lane & 16;
        const float send = up ? v[i] : v[i + 8];
        const float keep = up ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = lane & 8;
        const float send = up ? v[i] : v[i + 4];
        const float keep = up ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 4;
        const float send = up ? v[i] : v[i + 2];
        const float keep = up ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool up = lane & 2;
        const float send = up ? v[0] : v[1];
        const float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// kWin: the window form (a compile-time switch, so that the whole-matrix form
// keeps its registers)
template <bool kWin>
__global__ void __launch_bounds__(kGThreads, 1) gram_rbf_kernel(const __grid_constant__ CUtensorMap mapX, GramArgs g) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t bar_base = base + kGStages * kGStageBytes;
    auto full_bar = [&](int s) { return bar_base + 8u * s; };
    auto empty_bar = [&](int s) { return bar_base + 8u * (kGStages + s); };
    auto tfull_bar = [&](int b) { return bar_base + 8u * (2 * kGStages + b); };
    auto tempty_bar = [&](int b) { return bar_base + 8u * (2 * kGStages + 2 + b); };
    const uint32_t abort_bar = bar_base + 8u * (2 * kGStages + 4);
    uint8_t *misc = gbase + kGStages * kGStageBytes + 8 * (2 * kGStages + 5);   // inside kGBarBytes
    volatile uint32_t *tmem_holder = (volatile uint32_t *)misc;
    volatile int *abort_flag = (volatile int *)(misc + 4);
    volatile uint32_t *issued_cnt = (volatile uint32_t *)(misc + 8);
    volatile uint32_t *consumed_cnt = (volatile uint32_t *)(misc + 12);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = g.n;
    const int T = (int)((n + kGT - 1) / kGT);
    constexpr bool win = kWin;
    const int tm0 = win ? (int)(g.row0 / kGT) : 0, tn0 = win ? (int)(g.col0 / kGT) : 0;
    const int TN = win ? (int)((g.cols + kGT - 1) / kGT) : 0;
    const int total = win ? (int)((g.rows + kGT - 1) / kGT) * TN : T * (T + 1) / 2;
    const int64_t jend = win ? g.row0 + g.rows : n, kend = win ? g.col0 + g.cols : n;
    auto tile_of = [&](int t, int &tm, int &tn) {
        if (win) {
            tm = tm0 + t / TN;
            tn = tn0 + t % TN;
        } else {
            upper_tile(t, T, tm, tn);
        }
    };
    // Work units: whole tiles, except that the tiles of a last partial wave of at
    // most half the grid are split into column halves (64 columns each), so that
    // the last wave takes half a tile's time (whole-matrix form only; the counts
    // come with the arguments).
    const int units = win ? total : g.units;
    auto unit_of = [&](int u, int &tm, int &tn, int &c_off) {
        if (win || u < g.nfull) {
            tile_of(u, tm, tn);
            c_off = -1;   // whole tile
        } else {
            tile_of(g.nfull + ((u - g.nfull) >> 1), tm, tn);
            c_off = ((u - g.nfull) & 1) * (kGT / 2);
        }
    };
    const long long wlim = g.wait_limit > 0 ? g.wait_limit : kGWaitLimit;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGStages; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), kGEpiWarps);
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
                     "r"(kGTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: the tile's row block and column block of X
            uint32_t it = 0;
            for (int u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x) {
                int tm, tn, c_off;
                unit_of(u, tm, tn, c_off);   // a half loads the whole column block
                for (int kb = 0; kb < g.num_k; ++kb, ++it) {
                    const int s = it % kGStages;
                    if (it >= (uint32_t)kGStages && !mbar_wait(empty_bar(s), ((it / kGStages) - 1) & 1, abort_flag, wlim))
                        break;
                    const uint32_t sa = base + s * kGStageBytes;
                    mbar_expect_tx(full_bar(s), kGStageBytes);
                    tma_load_3d(sa, &mapX, kb * kGBK, tm * kGT, 0, full_bar(s));
                    tma_load_3d(sa + kGP * kGTile, &mapX, kb * kGBK, tn * kGT, 0, full_bar(s));
                    *issued_cnt = it + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            constexpr uint32_t idesc_full = make_idesc(1u, kGT, kGT);
            constexpr uint32_t idesc_half = make_idesc(1u, kGT, kGT / 2);
            uint32_t it = 0, tcount = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
                int tm, tn, c_off;
                unit_of(u, tm, tn, c_off);
                const uint32_t idesc = c_off < 0 ? idesc_full : idesc_half;
                // a half multiplies rows c_off .. c_off + 63 of the column block
                // (whole 8-row swizzle atoms: 64 rows x 64 bytes further on)
                const uint32_t b_row = c_off < 0 ? 0u : (uint32_t)c_off * kGRowBytes;
                const int buf = tcount & 1;
                if (tcount >= 2 && !mbar_wait(tempty_bar(buf), ((tcount >> 1) - 1) & 1, abort_flag, wlim)) break;
                tc_fence_after();
                // a half's accumulators sit at its own columns c_off .. c_off + 63
                const uint32_t d_hi = tmem + buf * kGAccCols + (c_off < 0 ? 0u : (uint32_t)c_off), d_lo = d_hi + kGT;
                for (int kb = 0; kb < g.num_k; ++kb, ++it) {
                    const int s = it % kGStages;
                    if (!mbar_wait(full_bar(s), (it / kGStages) & 1, abort_flag, wlim)) {
                        ok = false;
                        break;
                    }
                    *consumed_cnt = it + 1;
                    tc_fence_after();
                    const uint32_t sa = base + s * kGStageBytes, sb = sa + kGP * kGTile + b_row;
#pragma unroll
                    for (int kk = 0; kk < kGBK / 16; ++kk) {
                        uint64_t ad[kGP], bd[kGP];
#pragma unroll
                        for (int p = 0; p < kGP; ++p) {
                            ad[p] = desc_sw<kGRowBytes>(sa + p * kGTile + kk * 32);
                            bd[p] = desc_sw<kGRowBytes>(sb + p * kGTile + kk * 32);
                        }
                        const uint32_t acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
                        mma<false>(d_hi, ad[0], bd[0], idesc, acc0);
                        // every digit pair of weight 2^-8 .. 2^-24 into the second accumulator
                        mma<false>(d_lo, ad[0], bd[1], idesc, acc0);
#pragma unroll
                        for (int sum = 1; sum < kGP; ++sum) {
#pragma unroll
                            for (int i = 0; i <= sum; ++i) {
                                if (sum == 1 && i == 0) continue;   // issued above
                                mma<false>(d_lo, ad[i], bd[sum - i], idesc, 1u);
                            }
                        }
                    }
                    mma_commit(empty_bar(s));
                }
                if (!ok) break;
                mma_commit(tfull_bar(buf));
                ++tcount;
            }
        }
    } else {
        // ---------------- epilogue: warp w covers TMEM lanes 32 (w % 4) .. and 32
        // columns (2 chunks of 16) of the tile.  Each warp stages its 32 x 16 chunk
        // in shared memory, so that every global store writes whole 16-byte pieces
        // of consecutive addresses: the tile's rows (K and digit planes) and, off
        // the diagonal, the mirror rows of the digit planes.
        const int q = warp & 3;
        const int cg = (warp - 2) >> 2;
        const int ew = warp - 2;                 // epilogue warp 0..15
        EpiStage &stg = reinterpret_cast<EpiStage *>(gbase + kGStages * kGStageBytes + kGBarBytes)[ew];
        const float lead_scale = __int_as_float((127 + g.lead_k) << 23);   // 2^w of K's digits
        const float cscale = __int_as_float((127 + 1 - 2 * g.lead_x) << 23);   // 2^(1 - 2 w_x)
        double tot[kGMaxRed] = {0.0, 0.0, 0.0, 0.0};
        uint32_t tcount = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x) {
            int tm, tn, c_off;
            unit_of(u, tm, tn, c_off);
            const bool half = c_off >= 0;
            // the warp's columns (TMEM columns = tile columns): 32 (two chunks of 16)
            // of a whole tile, or 16 of a half
            const int wcol = half ? c_off + 16 * cg : 32 * cg;
            const int buf = tcount & 1;
            // the warp's column data (scale and squared norm of each column's x),
            // fetched while the accumulator may still be in flight
            {
                const int64_t k = (int64_t)tn * kGT + wcol + (half ? (lane & 15) : lane);   // arrays padded to whole tiles
                const float2 nk = g.nrm[k];
                const float4 cd = make_float4(g.sx[k] * cscale, nk.x, nk.y, 0.f);
                __syncwarp();   // the previous tile's column data are read
                stg.cd[lane] = cd;
            }
            int waited = 0;
            if (lane == 0) waited = mbar_wait(tfull_bar(buf), (tcount >> 1) & 1, abort_flag, wlim) ? 1 : 0;
            waited = __shfl_sync(0xffffffffu, waited, 0);
            __syncwarp();   // the column data are visible to the whole warp
            if (!waited || *abort_flag) break;
            tc_fence_after();
            const bool diag = tm == tn;
            const bool mirror = !win && !diag;   // the tile stands for its mirror too
            const int64_t j0 = (int64_t)tm * kGT + 32 * q;   // the warp's first row
            const int64_t j = j0 + lane;
            const bool jok = j < jend;
            const float sj = g.sx[j];
            const float2 nj = g.nrm[j];
            float rowsum[kGMaxRed] = {0.f, 0.f, 0.f, 0.f};
            float tsum[kGMaxRed] = {0.f, 0.f, 0.f, 0.f};
            const uint32_t taddr = tmem + buf * kGAccCols + ((uint32_t)(32 * q) << 16);
#pragma unroll 1
            for (int h = 0; h < (half ? 1 : 2); ++h) {
                const int c0 = wcol + 16 * h;   // tile column = TMEM column
                uint32_t hi[16], lo[16];
                tmem_ld16(taddr + c0, hi);
                tmem_ld16(taddr + kGT + c0, lo);
                tmem_wait_ld();
                const int64_t k0 = (int64_t)tn * kGT + c0;
                // squared distances: ||x_j||^2 + ||x_k||^2 - 2 x_j . x_k
                float v[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float4 ck = stg.cd[16 * h + c];
                    const float cf = sj * ck.x;                          // power of two
                    const float p = cf * __uint_as_float(hi[c]);         // exact
                    float s, es, tt, et2;
                    two_sum(nj.x, ck.y, s, es);
                    two_sum(s, -p, tt, et2);
                    const float d2 = tt + (((es + et2) + (nj.y + ck.z)) - cf * __uint_as_float(lo[c]));
                    v[c] = fmaxf(d2, 0.f);
                }
#pragma unroll
                for (int c = 0; c < 16; c += 2) {
                    float a, b;
                    f2_unpack(f2_rbf(f2_pack(v[c], v[c + 1]), g.inv_h), a, b);
                    v[c] = a, v[c + 1] = b;
                }
                const float dv = g.zero_diag ? 0.f : 1.f;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int64_t k = k0 + c;
                    if (k == j) v[c] = dv;
                    if (!jok || k >= kend) v[c] = 0.f;
                }
                // K: the warp's 32 tile rows through shared memory, 16-byte row pieces
#pragma unroll
                for (int c = 0; c < 16; ++c) stg.kf[lane][c] = v[c];
                __syncwarp();
                const bool kvec = (n & 3) == 0;
#pragma unroll
                for (int it = 0; it < 4; ++it) {
                    const int r = 8 * it + (lane >> 2), pc = lane & 3;
                    const int64_t jr = j0 + r, kc = k0 + 4 * pc;
                    if (jr < jend && (!kWin || g.K)) {
                        float *dst = g.K + jr * n + kc;
                        const float e0 = stg.kf[r][4 * pc], e1 = stg.kf[r][4 * pc + 1], e2 = stg.kf[r][4 * pc + 2],
                                    e3 = stg.kf[r][4 * pc + 3];
                        if (kvec && kc + 3 < kend) {
                            *reinterpret_cast<float4 *>(dst) = make_float4(e0, e1, e2, e3);
                        } else {
                            if (kc < kend) dst[0] = e0;
                            if (kc + 1 < kend) dst[1] = e1;
                            if (kc + 2 < kend) dst[2] = e2;
                            if (kc + 3 < kend) dst[3] = e3;
                        }
                    }
                }
                // the mirror of K, where K is read below the diagonal too: each store
                // writes 32 consecutive floats of a mirror row
                if (mirror && !g.upper_only && jok) {
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        if (k0 + c < n) g.K[(k0 + c) * n + j] = v[c];
                }
                // digit planes of K (row scale 1): y = K 2^w, digit p rounds y_p to a
                // multiple of 2^-8p (add and subtract 1.5 * 2^(23 - 8p)), exact
                if (g.slices) {
                    const int64_t plane = kWin ? g.splane : n * g.ldp;
                    float y[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) y[c] = v[c] * lead_scale;
                    float magic = 12582912.0f;   // 1.5 * 2^23
                    for (int p = 0; p < g.planes; ++p) {
                        uint32_t w[8];
#pragma unroll
                        for (int c = 0; c < 16; c += 2) {
                            const float d0 = (y[c] + magic) - magic, d1 = (y[c + 1] + magic) - magic;
                            y[c] -= d0;
                            y[c + 1] -= d1;
                            const __nv_bfloat162 b2 = __floats2bfloat162_rn(d0, d1);
                            w[c >> 1] = *reinterpret_cast<const uint32_t *>(&b2);
                        }
                        __syncwarp();   // the previous plane's pieces are read
#pragma unroll
                        for (int c2 = 0; c2 < 8; ++c2) stg.dr[lane][c2] = w[c2];
                        if (mirror) {
#pragma unroll
                            for (int c2 = 0; c2 < 8; ++c2) {
                                stg.dt[2 * c2][lane] = (unsigned short)(w[c2] & 0xffffu);
                                stg.dt[2 * c2 + 1][lane] = (unsigned short)(w[c2] >> 16);
                            }
                        }
                        __syncwarp();
                        __nv_bfloat16 *pl = g.slices + p * plane;
                        // tile rows: 32 B per row, two 16-byte pieces
                        if (k0 < g.ldp) {   // k0 is a multiple of 16 and ldp of 64
#pragma unroll
                            for (int it = 0; it < 2; ++it) {
                                const int r = 16 * it + (lane >> 1), pc = lane & 1;
                                const int64_t jr = j0 + r;
                                if (jr < jend)
                                    *reinterpret_cast<uint4 *>(pl + (kWin ? jr - g.srow0 : jr) * g.ldp + k0 + 8 * pc) =
                                        make_uint4(stg.dr[r][4 * pc], stg.dr[r][4 * pc + 1], stg.dr[r][4 * pc + 2],
                                                   stg.dr[r][4 * pc + 3]);
                            }
                        }
                        // mirror rows k0 .. k0 + 15, columns j0 .. j0 + 31: 64 B per row
                        if (mirror) {
#pragma unroll
                            for (int it = 0; it < 2; ++it) {
                                const int c = 8 * it + (lane >> 2), pc = lane & 3;
                                const int64_t kr = k0 + c;
                                if (kr < n && j0 + 8 * pc < n) {
                                    const uint4 pv = *reinterpret_cast<const uint4 *>(&stg.dt[c][8 * pc]);
                                    __nv_bfloat16 *dst = pl + kr * g.ldp + j0 + 8 * pc;
                                    if (j0 + 8 * pc + 7 < n) {
                                        *reinterpret_cast<uint4 *>(dst) = pv;
                                    } else {
                                        const unsigned short *e = reinterpret_cast<const unsigned short *>(&pv);
                                        for (int u = 0; u < 8; ++u)
                                            if (j0 + 8 * pc + u < n)
                                                reinterpret_cast<unsigned short *>(dst)[u] = e[u];
                                    }
                                }
                            }
                        }
                        magic *= (1.0f / 256.0f);
                    }
                    if ((win ? tn == tn0 : diag) && cg == 0 && h == 0 && jok && g.scales) g.scales[j] = 1.f;
                }
                __syncwarp();   // the staging buffers are free for the next chunk
                // fused reductions of entrywise powers of K
#pragma unroll
                for (int r = 0; r < kGMaxRed; ++r) {
                    if (r >= g.nred) break;
                    const int pw = g.red[r].pow;
                    float pv[16];
                    float sum = 0.f;
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        pv[c] = powk(v[c], pw);
                        sum += pv[c];
                    }
                    if (g.red[r].vec) {
                        rowsum[r] += sum;
                        if (mirror) {
                            // the mirror tile's rows: column sums of this tile
                            const float cs = transpose_reduce16(pv, lane);
                            const int col = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 +
                                            ((lane >> 1) & 1);
                            if ((lane & 1) == 0 && k0 + col < n) atomicAdd(g.red[r].out + k0 + col, (double)cs);
                        }
                    } else {
                        tsum[r] += sum;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(buf));
#pragma unroll
            for (int r = 0; r < kGMaxRed; ++r) {
                if (r >= g.nred) break;
                if (g.red[r].vec) {
                    if (jok) atomicAdd(g.red[r].out + j, (double)rowsum[r]);
                } else {
                    tot[r] += (double)tsum[r] * (mirror ? 2.0 : 1.0);
                }
            }
            ++tcount;
        }
#pragma unroll
        for (int r = 0; r < kGMaxRed; ++r) {
            if (r >= g.nred || g.red[r].vec) continue;
            const double s = warp_sum(tot[r]);
            if (lane == 0 && !*abort_flag) atomicAdd(g.red[r].out, s);
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (*abort_flag) {
        if (warp == 1 && lane == 0) {
            mma_commit(abort_bar);
            mbar_drain(abort_bar, 0, wlim);
        }
        if (threadIdx.x == 0) {
            if (g.err) atomicOr(g.err, kErrWordTimeout);
            for (uint32_t i = *consumed_cnt; i < *issued_cnt; ++i)
                if (!mbar_drain(full_bar(i % kGStages), (i / kGStages) & 1, wlim)) break;
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGTmemCols));
    }
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace

size_t kbuild_rbf_tc_scratch_bytes(int64_t n, int d) {
    const int64_t npad = round_up(n, kGT);
    const int64_t ldx = round_up(d, kGBK);
    return (size_t)round_up(npad * 4, 1024) + (size_t)round_up(npad * 8, 1024) +
           (size_t)round_up((int64_t)kGP * n * ldx * 2, 1024);
}

namespace {

// The scratch layout: X's row scales, squared norms and digit planes.
struct GramScratch {
    float *sx;
    float2 *nrm;
    __nv_bfloat16 *dig;
    int ldx, lead_x;
};

GramScratch gram_scratch(void *scratch, int64_t n, int d) {
    const int64_t npad = round_up(n, kGT);
    GramScratch r;
    r.ldx = (int)round_up(d, kGBK);
    r.lead_x = split_lead_bits(r.ldx);
    char *p = (char *)scratch;
    r.sx = (float *)p;
    p += round_up(npad * 4, 1024);
    r.nrm = (float2 *)p;
    p += round_up(npad * 8, 1024);
    r.dig = (__nv_bfloat16 *)p;
    return r;
}

cudaError_t gram_launch(const GramScratch &gs, int64_t n, double param, int zero_diag, float *K, void *slices,
                        int64_t ldp, int lead_bits, int planes, float *scales, int nred, const int *red_pow,
                        const int *red_vec, double *const *red_out, int upper_only, int64_t row0, int64_t rows,
                        int64_t col0, int64_t cols, int64_t srow0, int64_t splane, int *err, cudaStream_t s) {
    CUtensorMap map;
    if (!make_map_planes(&map, gs.dig, true, kGP, kGP, n, gs.ldx, kGT, kGRowBytes)) return cudaErrorInvalidValue;
    static std::atomic<bool> attr[64];   // per device, set once; atomic: host threads may launch concurrently
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(gram_rbf_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kGSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(gram_rbf_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    GramArgs g{};
    g.n = n;
    g.num_k = gs.ldx / kGBK;
    g.lead_x = gs.lead_x;
    g.sx = gs.sx;
    g.nrm = gs.nrm;
    g.inv_h = (float)(1.0 / param);
    g.zero_diag = zero_diag;
    g.K = K;
    g.upper_only = upper_only;
    g.slices = (__nv_bfloat16 *)slices;
    g.ldp = slices ? ldp : n;
    g.lead_k = lead_bits;
    g.planes = planes;
    g.scales = slices ? scales : nullptr;
    g.nred = nred;
    for (int q = 0; q < nred; ++q) {
        if (red_pow[q] < 1 || red_pow[q] > 4) return cudaErrorInvalidValue;
        g.red[q] = GramRed{red_pow[q], red_vec[q], red_out[q]};
    }
    g.err = err;
    g.wait_limit = tc_debug_wait_limit();
    g.row0 = row0;
    g.rows = rows;
    g.col0 = col0;
    g.cols = cols;
    g.srow0 = srow0;
    g.splane = splane > 0 ? splane : n * g.ldp;
    int64_t tiles;
    if (rows > 0) {
        tiles = ((rows + kGT - 1) / kGT) * ((cols + kGT - 1) / kGT);
    } else {
        const int64_t T = round_up(n, kGT) / kGT;
        tiles = T * (T + 1) / 2;
    }
    const int64_t S = sm_count();
    const int grid = (int)(tiles < S ? tiles : S);
    // the last partial wave in column halves where they fit in one wave
    const int last = rows > 0 ? 0 : (int)(tiles % grid);
    const bool split = last > 0 && 2 * last <= grid;
    g.nfull = (int)tiles - (split ? last : 0);
    g.units = g.nfull + (split ? 2 * last : 0);
    if (rows > 0) gram_rbf_kernel<true><<<grid, kGThreads, kGSmem, s>>>(map, g);
    else gram_rbf_kernel<false><<<grid, kGThreads, kGSmem, s>>>(map, g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gram_rbf_prep(const void *X, int x_dtype, int64_t n, int d, void *scratch, int *err,
                                 cudaStream_t s) {
    if (!X || !scratch || d < 1 || d > 8 * kGBK || ((uintptr_t)scratch % 256) != 0) return cudaErrorInvalidValue;
    const GramScratch gs = gram_scratch(scratch, n, d);
    const int64_t npad = round_up(n, kGT);
    gram_xsplit_kernel<<<(unsigned)((npad + 7) / 8), 256, 0, s>>>(X, x_dtype, n, npad, d, gs.ldx, gs.lead_x, gs.dig,
                                                                  gs.sx, gs.nrm, err);
    return cudaGetLastError();
}

cudaError_t launch_gram_rbf_window(int64_t n, int d, double param, int zero_diag, float *K, void *slices,
                                   int64_t ldp, int lead_bits, int planes, float *scales, int nred,
                                   const int *red_pow, const int *red_vec, double *const *red_out, int64_t row0,
                                   int64_t rows, int64_t col0, int64_t cols, int64_t srow0, int64_t splane,
                                   void *scratch, int *err, cudaStream_t s) {
    if (nred < 0 || nred > kGMaxRed || (slices && (planes < 3 || planes > 5)) || !scratch || d < 1 ||
        d > 8 * kGBK || ((uintptr_t)scratch % 256) != 0 || (slices && ldp % 64 != 0) || rows < 1 || cols < 1 ||
        row0 < 0 || col0 < 0 || row0 % kGT != 0 || col0 % kGT != 0 || row0 + rows > n || col0 + cols > n ||
        (slices && (srow0 > row0 || splane < (row0 + rows - srow0) * ldp)))
        return cudaErrorInvalidValue;
    return gram_launch(gram_scratch(scratch, n, d), n, param, zero_diag, K, slices, ldp, lead_bits, planes, scales,
                       nred, red_pow, red_vec, red_out, 0, row0, rows, col0, cols, srow0, splane, err, s);
}

cudaError_t launch_kbuild_rbf_tc(const void *X, int x_dtype, int64_t n, int d, double param, int zero_diag, float *K,
                                 void *slices, int64_t ldp, int lead_bits, int planes, float *scales, int nred,
                                 const int *red_pow, const int *red_vec, double *const *red_out, int upper_only,
                                 void *scratch, int *err, cudaStream_t s) {
    if (nred < 0 || nred > kGMaxRed || (slices && (planes < 3 || planes > 5)) || !X || !K || !scratch || d < 1 ||
        d > 8 * kGBK || ((uintptr_t)scratch % 256) != 0 || (slices && ldp % 64 != 0))
        return cudaErrorInvalidValue;
    cudaError_t e = launch_gram_rbf_prep(X, x_dtype, n, d, scratch, err, s);
    if (e != cudaSuccess) return e;
    return gram_launch(gram_scratch(scratch, n, d), n, param, zero_diag, K, slices, ldp, lead_bits, planes, scales,
                       nred, red_pow, red_vec, red_out, upper_only, 0, 0, 0, 0, 0, 0, err, s);
}

}  // namespace ustat
