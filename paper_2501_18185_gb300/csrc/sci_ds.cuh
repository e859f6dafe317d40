// Paired-FP32 ("double-single") arithmetic shared by the sigma kernels and the block-vector
// kernels.
//
// On GB300 the FP64 pipe runs 2 FMA per clock per SM against 128 FP32 operations, so
// FP64-accurate sums are carried on the FP32 pipes: a value x is held as hi + lo with
// hi, lo floats (48 significant bits).  For t = th + tl and c = ch + cl the product is
//     p = fl(th*ch),  e = (th*ch - p) + th*cl + tl*ch,
// the first term exact through one FMA and the dropped tl*cl about 2^-48 of |tc|; a sum
// (hi, lo) takes p by TwoSum (Knuth) and folds e and the rounding error into lo.
// Conversions between double and float pairs go through the integer pipes: the F2F
// conversion instructions share the narrow FP64 pipe.
#pragma once

#include <cstdint>

namespace sci {

struct Ds {
    float hi, lo;
};

__device__ __forceinline__ void ds_zero(Ds &a) { a.hi = 0.f, a.lo = 0.f; }

// a += t * c
__device__ __forceinline__ void ds_fma(Ds &a, float2 t, float2 c)
{
    const float p = t.x * c.x;
    float e = fmaf(t.x, c.x, -p);
    e = fmaf(t.x, c.y, e);
    e = fmaf(t.y, c.x, e);
    const float s = a.hi + p;
    const float bv = s - a.hi;
    const float err = (a.hi - (s - bv)) + (p - bv);
    a.lo += err + e;
    a.hi = s;
}

// a += b for a paired-FP32 value b = (hi, lo)
__device__ __forceinline__ void ds_add(Ds &a, float2 b)
{
    const float s = a.hi + b.x;
    const float bv = s - a.hi;
    const float err = (a.hi - (s - bv)) + (b.x - bv);
    a.lo += err + b.y;
    a.hi = s;
}

__device__ __forceinline__ void ds_renorm(Ds &a)
{
    const float s = a.hi + a.lo;
    a.lo = a.lo - (s - a.hi);
    a.hi = s;
}

// float -> double by bit assembly.  Normal numbers, zero, inf and NaN convert exactly; a
// float denormal (|x| < 1.2e-38) becomes a signed zero.
__device__ __forceinline__ double f2d_int(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    unsigned long long bits = sign;
    if (e == 0xFFu) bits |= (0x7FFull << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
    else if (e != 0u) bits |= ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double ds_value(Ds a) { return f2d_int(a.hi) + f2d_int(a.lo); }

// double -> (hi, lo) by bit manipulation: hi keeps the sign, the exponent and the leading
// 24 significant bits (truncated), lo the next 24 bits of the remainder, normalised with
// a count of leading zeros.  hi + lo equals x to a relative 2^-47.  |x| below 2^-126
// (1.2e-38) and remainders below it flush to zero; |x| at or above 2^128 cannot occur in
// the normalised vectors this serves and is passed through the FP64 conversion.
__device__ __forceinline__ float2 ds_split_int(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7FF);
    const int ef = e - 896;  // float biased exponent of hi
    if (ef >= 255) return make_float2((float)x, 0.f);
    if (ef <= 0) return make_float2(__uint_as_float(sign), 0.f);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    const float hi = __uint_as_float(sign | ((uint32_t)ef << 23) | (uint32_t)(m >> 29));
    const uint32_t r = (uint32_t)(m & 0x1FFFFFFFull);  // remainder: r * 2^(e - 1075)
    if (r == 0u) return make_float2(hi, 0.f);
    const int p = 31 - __clz((int)r);                   // leading one of r, 0..28
    const int el = p + e - 948;                         // float biased exponent of lo
    if (el <= 0) return make_float2(hi, 0.f);
    const uint32_t frac = (p >= 23 ? (r >> (p - 23)) : (r << (23 - p))) & 0x7FFFFFu;
    return make_float2(hi, __uint_as_float(sign | ((uint32_t)el << 23) | frac));
}

}  // namespace sci
