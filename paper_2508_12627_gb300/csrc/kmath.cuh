// Number formats shared by the kernels: the split-bf16 fixed-point digits of an
// operand row, packed float32 pair arithmetic (.f32x2), and the RBF kernel map
// exp(-d2 / h) in float32 with an unbiased exponential.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ustat {

__device__ __forceinline__ int row_exp(float m) {
    // smallest e with m <= 2^e (m = f 2^e, f in [0.5, 1); f = 0.5 means m = 2^(e-1))
    int e = 0;
    if (m > 0.f) {
        const float f = frexpf(m, &e);
        if (f == 0.5f) e -= 1;
    }
    return e;
}

__device__ __forceinline__ int row_exp(double m) {
    int e = 0;
    if (m > 0.0) {
        const double f = frexp(m, &e);
        if (f == 0.5) e -= 1;
    }
    return e;
}

// float64 source (the wide-storage mode), digits of the value itself rather than
// of its float32 rounding.  y = x 2^(w - e) (|y| <= 2^w) is rounded once to a
// multiple of 2^-8(planes - 1), as the integer q; its balanced base-256 digits
// (each in [-128, 127], the leading one |d1| <= 2^w) are taken with integer
// arithmetic: no float64 arithmetic per entry (this part's float64 pipe runs at
// a small fraction of its float32 and integer rates).
// rint(x 2^k), ties to even as llrint, for a float64 x with |x 2^k| < 2^53: the
// integer mantissa shifted right with the round bit taken from the bits shifted
// out (integer operations only); the arithmetic route for what this does not
// cover (not finite, or a left shift).
__device__ __forceinline__ long long rint_scaled(double x, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 2047u);
    unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (ex != 0) m |= 1ull << 52;
    const int sh = 1075 - k - (ex != 0 ? ex : 1);   // x 2^k = m 2^-sh
    if (ex == 2047 || sh < 0) return llrint(ldexp(x, k));
    unsigned long long q = 0;
    if (sh == 0) {
        q = m;
    } else if (sh < 64) {
        q = m >> sh;
        const unsigned long long r = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (r > half || (r == half && (q & 1ull))) ++q;
    }
    return (b >> 63) ? -(long long)q : (long long)q;
}

__device__ __forceinline__ void write_digits(double x, int lead_bits, int e, int planes, __nv_bfloat16 *dst,
                                             int64_t plane_stride) {
    long long q = rint_scaled(x, lead_bits - e + 8 * (planes - 1));   // the scaling is exact
    float scale = __int_as_float((127 - 8 * (planes - 1)) << 23);       // 2^-8(planes - 1)
    for (int p = planes - 1; p >= 1; --p) {
        const int dp = (int)(((q + 128) & 255) - 128);
        q = (q - dp) >> 8;                                               // exact
        dst[p * plane_stride] = __float2bfloat16_rn((float)dp * scale);   // exact
        scale *= 256.f;
    }
    dst[0] = __float2bfloat16_rn((float)q);                              // |q| <= 2^w: exact
}

__device__ __forceinline__ void write_digits(float x, int lead_bits, int e, int planes, __nv_bfloat16 *dst,
                                             int64_t plane_stride) {
    const int k = lead_bits - e;
    float y = (k >= -126 && k <= 127) ? x * __int_as_float((127 + k) << 23) : ldexpf(x, k);   // |y| <= 2^w, exact
    float d = rintf(y);
    dst[0] = __float2bfloat16_rn(d);
    float scale = 1.f / 256.f;
    for (int p = 1; p < planes; ++p) {
        y = (y - d) * 256.f;              // exact
        d = rintf(y);
        dst[p * plane_stride] = __float2bfloat16_rn(d * scale);
        scale *= (1.f / 256.f);
    }
}

// x 2^e as a float64, for a float32 x, by assembling the float64's bit fields:
// integer operations only, exact (the float32 mantissa fits).  The arithmetic
// route (conversion, then scaling) handles what the bit route does not: zero,
// a float32 subnormal, infinity or NaN, or a result outside the normal float64
// range.
__device__ __forceinline__ double f2d_scaled(float x, int e) {
    const uint32_t b = __float_as_uint(x);
    const int ex = (int)((b >> 23) & 255u);
    const int de = ex + (1023 - 127) + e;
    if (ex == 0 || ex == 255 || de <= 0 || de >= 2047) return x == 0.f ? 0.0 : ldexp((double)x, e);
    const uint32_t hw = (b & 0x80000000u) | ((uint32_t)de << 20) | ((b & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hw, (int)(b << 29));
}

// The float32 nearest to x (ties to even), by integer operations on the bit
// fields: the 52-bit significand is cut to 23 bits and rounded up when the cut
// part is above half a unit, or exactly half with an odd kept part; a carry out
// of the significand moves into the exponent (up to infinity above the largest
// float).  Zeros and values outside float32's normal range (subnormal results,
// infinities, NaN) take the float64 conversion.
__device__ __forceinline__ float d2f_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32);
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023;
    if (e < -126 || e > 127) return (float)x;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    uint32_t f = ((uint32_t)(e + 127) << 23) | (uint32_t)(m >> 29);
    const uint32_t cut = (uint32_t)(m & 0x1FFFFFFFull), half = 0x10000000u;
    f += (cut > half || (cut == half && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f | (hi & 0x80000000u));
}

// s + t = a + b exactly, s = fl(a + b) (Knuth's TwoSum, six float32 operations)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// two float32 in one 64-bit register pair (first = low half)
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_pack(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f32x2 f2_splat(float a) { return f2_pack(a, a); }
__device__ __forceinline__ f32x2 f2_rint(f32x2 a) {
    float x, y;
    f2_unpack(a, x, y);
    return f2_pack(rintf(x), rintf(y));
}

// exp(-d2 * inv_h) for two squared distances: the steps of exp_unbiased, each
// the same IEEE operation per lane
__device__ __forceinline__ f32x2 f2_rbf(f32x2 d2, float inv_h) {
    const f32x2 z = f2_mul(d2, f2_splat(-inv_h));
    const f32x2 k = f2_rint(f2_mul(z, f2_splat(1.44269504088896341f)));
    const f32x2 fh = f2_fma(k, f2_splat(-0.693145751953125f), z);   // exact
    const f32x2 fl = f2_mul(k, f2_splat(-1.42860682030941723212e-6f));
    const f32x2 f = f2_add(fh, fl);
    f32x2 q = f2_fma(f2_splat(1.0f / 40320.0f), f, f2_splat(1.0f / 5040.0f));
    q = f2_fma(q, f, f2_splat(1.0f / 720.0f));
    q = f2_fma(q, f, f2_splat(1.0f / 120.0f));
    q = f2_fma(q, f, f2_splat(1.0f / 24.0f));
    q = f2_fma(q, f, f2_splat(1.0f / 6.0f));
    q = f2_fma(q, f, f2_splat(0.5f));
    q = f2_mul(f2_mul(q, f), f);
    const f32x2 one = f2_splat(1.0f);
    const f32x2 sh = f2_add(one, fh);                        // Fast2Sum (|1| >= |fh|)
    const f32x2 sl = f2_sub(fh, f2_sub(sh, one));
    const f32x2 y = f2_add(sh, f2_add(f2_add(sl, fl), q));
    float k0, k1, z0, z1;
    f2_unpack(k, k0, k1);
    f2_unpack(z, z0, z1);
    const f32x2 p2 = f2_pack(__int_as_float(((int)k0 + 127) << 23), __int_as_float(((int)k1 + 127) << 23));
    float r0, r1;
    f2_unpack(f2_mul(y, p2), r0, r1);
    return f2_pack(z0 < -87.0f ? 0.0f : r0, z1 < -87.0f ? 0.0f : r1);
}

}  // namespace ustat
