// Tensor-core (tcgen05 + TMA, sm_103a) form of the s = 2 elimination step
// (Appendix D: summing out an index with two live neighbours is the matrix
// product C(j, k) = sum_i A(i, j) u(i) B(i, k)), with either a stored C or the
// fused reduction sum_jk C(j, k) W(j, k) a(j) b(k) of a component's last step.
//
// BF16X3 mode.  Each K-major operand row X(j, .) is written as three bf16
// fixed-point slices relative to a power-of-two row scale s_j >= max |X(j, .)|:
//     X(j, i) = s_j 2^-w (d1 + d2 2^-8 + d3 2^-16),  d1 in [-2^w, 2^w], |d2|,|d3| <= 128
// with hi = d1 (an integer), mid = d2 2^-8, lo = d3 2^-16, each exact in bf16.
// The product of two rows is accumulated as
//     ACC_hi = sum_i hi_A hi_B                          (integers, exact in FP32
//                                                        because n 4^w <= 2^24)
//     ACC_lo = sum_i (hi mid + mid hi + hi lo + lo hi + mid mid)
// and C = s_j s_k 2^-2w (ACC_hi + ACC_lo).  The dropped terms (mid lo, lo mid,
// lo lo) are below 2^-24 of the leading product.  Exact accumulation of the
// leading term removes the rounding bias of the tensor cores' FP32 accumulator,
// which otherwise does not average out over the n^2 terms of a V-statistic.
//
// TF32 mode: one tf32 operand copy (rounded to nearest), one accumulator.
//
// Kernel structure: one 128 x 128 output tile per CTA, 128 threads.  Thread 0
// issues TMA loads into a 2- or 4-stage ring (128-byte swizzle), thread 32
// issues the MMAs into TMEM (cta_group::1, M = 128, N = 128), then all four
// warps drain their 32 TMEM lanes with tcgen05.ld for the epilogue.  Every
// mbarrier wait is bounded; on time-out the CTA records an error, waits (again
// bounded) for its own copies in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "kcommon.cuh"
#include "kernels.h"

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

// One block per 32 operand rows j.  Pass 1: row maxima |X(j, i)| over all i.
// Pass 2: digits, written K-major through a shared-memory transpose when the
// source is read along columns.
template <bool kSplit>
__global__ void __launch_bounds__(256) operand_kernel(const float *__restrict__ M, int trans,
                                                      const double *__restrict__ u, int64_t n, int64_t ldp,
                                                      int lead_bits, __nv_bfloat16 *__restrict__ slices,
                                                      float *__restrict__ scales, float *__restrict__ prep) {
    __shared__ float tile[32][33];
    __shared__ float rmax[8][32];
    __shared__ int rexp[32];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    // X(j, i) = M[i][j] u(i) (trans = 0: column j of M) or M[j][i] u(i) (trans = 1)
    auto val = [&](int64_t j, int64_t i) -> float {
        if (j >= n || i >= n) return 0.f;
        float x = trans ? M[j * n + i] : M[i * n + j];
        if (u) x *= (float)u[i];
        return x;
    };
    int e_row = 0;
    if (kSplit) {
        float mx = 0.f;   // thread handles column j0 + tx (trans = 0) or row-major reads
        if (!trans) {
            for (int64_t i = ty; i < n; i += 8) mx = fmaxf(mx, fabsf(val(j0 + tx, i)));
            rmax[ty][tx] = mx;
        } else {
            // rows j0 + ty + 8 r, lanes walk i
            for (int r = 0; r < 4; ++r) {
                float m2 = 0.f;
                for (int64_t i = tx; i < n; i += 32) m2 = fmaxf(m2, fabsf(val(j0 + ty + 8 * r, i)));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
                if (tx == 0) tile[ty + 8 * r][0] = m2;
            }
        }
        __syncthreads();
        if (ty == 0) {
            float m = 0.f;
            if (!trans) {
                for (int q = 0; q < 8; ++q) m = fmaxf(m, rmax[q][tx]);
            } else {
                m = tile[tx][0];
            }
            int e = 0;
            if (m > 0.f) {
                // smallest e with m <= 2^e (m = f 2^e, f in [0.5, 1); f = 0.5 means m = 2^(e-1))
                const float f = frexpf(m, &e);
                if (f == 0.5f) e -= 1;
            }
            rexp[tx] = e;
            if (j0 + tx < n) scales[j0 + tx] = ldexpf(1.f, e);
        }
        __syncthreads();
    }
    (void)e_row;
    const int64_t plane = n * ldp;
    for (int64_t i0 = 0; i0 < ldp; i0 += 32) {
        // gather X(j0 + jj, i0 + ii) into tile[jj][ii]
        if (!trans) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                int ii = ty + 8 * r;
                tile[tx][ii] = val(j0 + tx, i0 + ii);   // coalesced along j (tx)
            }
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                int jj = ty + 8 * r;
                tile[jj][tx] = val(j0 + jj, i0 + tx);   // coalesced along i (tx)
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int jj = ty + 8 * r;
            const int64_t j = j0 + jj, i = i0 + tx;
            if (j >= n) continue;
            const float x = tile[jj][tx];
            if (kSplit) {
                const float y = ldexpf(x, lead_bits - rexp[jj]);   // |y| < 2^w, exact
                const float d1 = rintf(y);
                const float y2 = (y - d1) * 256.f;                  // exact
                const float d2 = rintf(y2);
                const float d3 = rintf((y2 - d2) * 256.f);
                const int64_t o = j * ldp + i;
                slices[o] = __float2bfloat16_rn(d1);
                slices[plane + o] = __float2bfloat16_rn(d2 * (1.f / 256.f));
                slices[2 * plane + o] = __float2bfloat16_rn(d3 * (1.f / 65536.f));
            } else {
                uint32_t t;
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
                prep[j * ldp + i] = __uint_as_float(t);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after ~2^22 polls with back-off (well over a second) or
// as soon as another thread of the CTA has given up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (it > 64) __nanosleep(256);
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major tile, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // SBO
    d |= (uint64_t)1 << 46;             // version
    d |= (uint64_t)2 << 61;             // SWIZZLE_128B
    return d;
}

template <int kKind>   // 0 = f16 (bf16 inputs), 1 = tf32
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if (kKind == 0)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

#define USTAT_R16(x) \
    "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]), "=r"(x[7]), "=r"(x[8]), \
        "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]), "=r"(x[13]), "=r"(x[14]), "=r"(x[15])

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : USTAT_R16(r)
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Instruction descriptor: D = F32, A/B format (1 = BF16 for kind::f16, 2 = TF32),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

constexpr int kBM = 128, kBN = 128;

template <int kKind>
struct TcCfg;
template <>
struct TcCfg<0> {   // bf16x3: 64 bf16 (128 B) per row per stage, 3 planes
    static constexpr int kBKElems = 64;
    static constexpr int kPlanes = 3;
    static constexpr int kStages = 2;
    static constexpr int kTileBytes = kBM * 128;                 // one plane tile
    static constexpr int kStageBytes = 2 * kPlanes * kTileBytes; // A + B
    static constexpr int kTmemCols = 256;                        // hi + lo accumulators
    static constexpr int kMmaK = 16;
};
template <>
struct TcCfg<1> {   // tf32: 32 floats (128 B) per row per stage
    static constexpr int kBKElems = 32;
    static constexpr int kPlanes = 1;
    static constexpr int kStages = 4;
    static constexpr int kTileBytes = kBM * 128;
    static constexpr int kStageBytes = 2 * kPlanes * kTileBytes;
    static constexpr int kTmemCols = 128;
    static constexpr int kMmaK = 8;
};

template <int kKind>
constexpr int tc_smem_bytes() {
    return TcCfg<kKind>::kStages * TcCfg<kKind>::kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
}

template <int kKind>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcGemmArgs g) {
    using Cfg = TcCfg<kKind>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t bar_base = base + Cfg::kStages * Cfg::kStageBytes;
    auto full_bar = [&](int s) { return bar_base + 8u * s; };
    auto empty_bar = [&](int s) { return bar_base + 8u * (Cfg::kStages + s); };
    const uint32_t done_bar = bar_base + 8u * (2 * Cfg::kStages);
    volatile uint32_t *tmem_holder = (volatile uint32_t *)(gbase + Cfg::kStages * Cfg::kStageBytes + 8 * (2 * Cfg::kStages + 1));
    volatile int *abort_flag = (volatile int *)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.y * kBM, n0 = (int64_t)blockIdx.x * kBN;
    const int num_k = (int)(g.ldp / Cfg::kBKElems);

    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::kStages; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void *)tmem_holder)),
                     "r"(Cfg::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    int issued = 0;   // producer: number of k-blocks whose loads were issued
    if (threadIdx.x == 0) {
        // ---------------- TMA producer
        for (int kb = 0; kb < num_k; ++kb) {
            const int s = kb % Cfg::kStages;
            if (kb >= Cfg::kStages) {
                if (!mbar_wait(empty_bar(s), ((kb / Cfg::kStages) - 1) & 1, abort_flag)) break;
            }
            const uint32_t sa = base + s * Cfg::kStageBytes;
            const uint32_t sb = sa + Cfg::kPlanes * Cfg::kTileBytes;
            mbar_expect_tx(full_bar(s), Cfg::kStageBytes);
            const int kc = kb * Cfg::kBKElems;
            tma_load_3d(sa, &mapA, kc, (int)m0, 0, full_bar(s));
            tma_load_3d(sb, &mapB, kc, (int)n0, 0, full_bar(s));
            issued = kb + 1;
        }
    } else if (threadIdx.x == 32) {
        // ---------------- MMA issuer
        constexpr uint32_t idesc = make_idesc(kKind == 0 ? 1u : 2u, kBM, kBN);
        const uint32_t d_hi = tmem, d_lo = tmem + 128;
        bool ok = true;
        for (int kb = 0; kb < num_k && ok; ++kb) {
            const int s = kb % Cfg::kStages;
            if (!mbar_wait(full_bar(s), (kb / Cfg::kStages) & 1, abort_flag)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = base + s * Cfg::kStageBytes;
            const uint32_t sb = sa + Cfg::kPlanes * Cfg::kTileBytes;
#pragma unroll
            for (int kk = 0; kk < Cfg::kBKElems / Cfg::kMmaK; ++kk) {
                const uint32_t koff = kk * Cfg::kMmaK * (kKind == 0 ? 2 : 4);   // bytes along K
                const uint32_t acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
                if (kKind == 0) {
                    const uint64_t ah = desc_sw128(sa + koff), am = desc_sw128(sa + Cfg::kTileBytes + koff),
                                   al = desc_sw128(sa + 2 * Cfg::kTileBytes + koff);
                    const uint64_t bh = desc_sw128(sb + koff), bm = desc_sw128(sb + Cfg::kTileBytes + koff),
                                   bl = desc_sw128(sb + 2 * Cfg::kTileBytes + koff);
                    mma<0>(d_hi, ah, bh, idesc, acc0);
                    mma<0>(d_lo, ah, bm, idesc, acc0);
                    mma<0>(d_lo, am, bh, idesc, 1u);
                    mma<0>(d_lo, ah, bl, idesc, 1u);
                    mma<0>(d_lo, al, bh, idesc, 1u);
                    mma<0>(d_lo, am, bm, idesc, 1u);
                } else {
                    mma<1>(d_hi, desc_sw128(sa + koff), desc_sw128(sb + koff), idesc, acc0);
                }
            }
            mma_commit(empty_bar(s));   // frees the stage when these MMAs complete
        }
        mma_commit(done_bar);           // accumulators final (or the loop gave up)
    }
    __syncwarp();

    // ---------------- epilogue: warp w owns TMEM lanes (tile rows) 32w .. 32w + 31
    const bool waited = mbar_wait(done_bar, 0, abort_flag);
    // tcgen05.ld is warp-collective: decide per warp
    const bool good = __all_sync(0xffffffffu, waited && !*abort_flag);
    tc_fence_after();
    const int64_t j = m0 + warp * 32 + lane;
    double red = 0.0;
    if (good) {
        const float rs = (j < g.n) ? ((kKind == 0) ? ldexpf(g.scaleA[j], -2 * g.lead_bits) : 1.f) : 0.f;
        const float aj = (g.a && j < g.n) ? (float)g.a[j] : 1.f;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < kBN; c0 += 16) {
            uint32_t hi[16], lo[16];
            tmem_ld16(lane_addr + c0, hi);
            if (kKind == 0) tmem_ld16(lane_addr + 128 + c0, lo);
            tmem_wait_ld();
            float part = 0.f;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int64_t k = n0 + c0 + c;
                float v = __uint_as_float(hi[c]);
                if (kKind == 0) v = (v + __uint_as_float(lo[c])) * g.scaleB[k < g.n ? k : 0];
                v *= rs;
                if (g.C) {
                    if (j < g.n && k < g.n) g.C[j * g.n + k] = v;
                } else if (j < g.n && k < g.n) {
                    float w = g.b ? (float)g.b[k] : 1.f;
                    if (g.W) w *= g.transW ? g.W[k * g.n + j] : g.W[j * g.n + k];
                    part = fmaf(v, w, part);
                }
            }
            red += (double)part;
        }
        red *= (double)aj;
    }
    const bool failed = __syncthreads_or(!good);
    if (failed) {
        if (threadIdx.x == 0 && g.err) atomicExch(g.err, 1);
        // wait (bounded) for this CTA's copies in flight before the smem goes away
        if (threadIdx.x == 0) {
            volatile int dummy = 0;
            for (int kb = 0; kb < issued; ++kb) {
                const int s = kb % Cfg::kStages;
                // a stage is in flight if it was issued and never consumed; try each once
                for (int it = 0; it < (1 << 20); ++it)
                    if (mbar_try_wait(full_bar(s), (kb / Cfg::kStages) & 1)) break;
            }
            (void)dummy;
        }
    }
    if (!g.C) {
        red = block_sum(red);
        if (threadIdx.x == 0 && !failed) atomicAdd(g.red, red);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kTmemCols));
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

// planes x rows x ldp (innermost) tensor, box {128 bytes, 128 rows, planes}.
bool make_map(CUtensorMap *map, const void *ptr, bool bf16, int planes, int64_t rows, int64_t ldp) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return false;
    const int esz = bf16 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)ldp, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)(ldp * esz), (cuuint64_t)(rows * ldp * esz)};
    cuuint32_t box[3] = {(cuuint32_t)(128 / esz), 128u, (cuuint32_t)planes};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                     const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int kKind>
cudaError_t launch_tc(const TcGemmArgs &g, cudaStream_t s) {
    CUtensorMap ma, mb;
    const bool bf16 = kKind == 0;
    const int planes = bf16 ? 3 : 1;
    if (!make_map(&ma, g.opA, bf16, planes, g.n, g.ldp) || !make_map(&mb, g.opB, bf16, planes, g.n, g.ldp))
        return cudaErrorInvalidValue;
    constexpr int smem = tc_smem_bytes<kKind>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<kKind>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((unsigned)((g.n + kBN - 1) / kBN), (unsigned)((g.n + kBM - 1) / kBM));
    tc_gemm_kernel<kKind><<<grid, 128, smem, s>>>(ma, mb, g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_split(const float *M, int trans, const double *u, int64_t n, int64_t ldp, int lead_bits,
                         void *slices, float *scales, cudaStream_t s) {
    dim3 grid((unsigned)((n + 31) / 32)), block(32, 8);
    operand_kernel<true><<<grid, block, 0, s>>>(M, trans, u, n, ldp, lead_bits, (__nv_bfloat16 *)slices, scales,
                                                nullptr);
    return cudaGetLastError();
}

cudaError_t launch_prep(const float *M, int trans, const double *u, int64_t n, int64_t ldp, float *out,
                        cudaStream_t s) {
    dim3 grid((unsigned)((n + 31) / 32)), block(32, 8);
    operand_kernel<false><<<grid, block, 0, s>>>(M, trans, u, n, ldp, 0, nullptr, nullptr, out);
    return cudaGetLastError();
}

cudaError_t launch_gemm_bf16x3(const TcGemmArgs &g, cudaStream_t s) { return launch_tc<0>(g, s); }
cudaError_t launch_gemm_tf32(const TcGemmArgs &g, cudaStream_t s) { return launch_tc<1>(g, s); }

}  // namespace ustat
