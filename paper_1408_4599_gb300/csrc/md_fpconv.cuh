// md_fpconv.cuh -- FP32 <-> FP64 conversions, k + 1/2 as a double and the
// floor of a double written as integer bit operations.
//
// GB300 executes the hardware conversions (float <-> double, int <->
// double) on its FP64 pipe, which runs at a small fraction of the FP32
// rate, and the integrator and the rebuild are bound by that pipe.  These forms run on the
// integer pipes instead and give the same bits as the hardware's
// round-to-nearest-even conversions under flush-to-zero, with one stated
// exception each (d2f_bits: values below FLT_MIN, floor_bits: NaN).  Plain
// C++ apart from the bit casts, so that a host program can check them
// against the CPU's IEEE-754 conversions.
#pragma once

#include <stdint.h>
#if defined(__CUDACC__)
#define MD_HD __host__ __device__ __forceinline__
#else
#include <string.h>
#define MD_HD inline
#endif

namespace mdk {

MD_HD uint64_t dbits(double x)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    return u;
#endif
}

MD_HD double bitsd(uint64_t u)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, sizeof x);
    return x;
#endif
}

MD_HD uint32_t fbits(float x)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(x);
#else
    uint32_t u;
    memcpy(&u, &x, sizeof u);
    return u;
#endif
}

MD_HD float bitsf(uint32_t u)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float x;
    memcpy(&x, &u, sizeof x);
    return x;
#endif
}

// (double)f, exact: the exponent rebased from 127 to 1023, the 23-bit
// fraction placed at the top of the 52-bit one.  Zeros and subnormal inputs
// give a signed zero (flush-to-zero), infinities and NaNs stay so.
MD_HD double f2d_bits(float f)
{
    const uint32_t u = fbits(f);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    if (e == 0) return bitsd(sign);
    const uint64_t ed = e == 0xffu ? 0x7ffu : (uint64_t)e + (1023u - 127u);
    return bitsd(sign | (ed << 52) | ((uint64_t)(u & 0x7fffffu) << 29));
}

// (float)x rounded to nearest, ties to even: the 52-bit fraction cut to 23
// bits with the exponent rebased (a carry out of the fraction moves to the
// next binade, and past the largest float to infinity).  |x| below FLT_MIN
// gives a signed zero (flush-to-zero; unlike the hardware, also in the
// sliver just below FLT_MIN that rounds up to it); NaN gives the canonical
// quiet NaN.
MD_HD float d2f_bits(double x)
{
    const uint64_t u = dbits(x);
    const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
    const uint64_t a = u & 0x7fffffffffffffffull;
    if (a < (uint64_t)(1023u - 126u) << 52) return bitsf(sign);
    if (a > 0x7ff0000000000000ull) return bitsf(0x7fffffffu);
    if (a >= (uint64_t)(1023u + 128u) << 52) return bitsf(sign | 0x7f800000u);  // |x| >= 2^128
    uint32_t r = (uint32_t)((a >> 29) - ((uint64_t)(1023u - 127u) << 23));
    const uint32_t rem = (uint32_t)a & 0x1fffffffu;
    r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;  // at most 0x7f800000: infinity
    return bitsf(sign | r);
}

// k + 1/2 as a double, exact, for 0 <= k < 2^30: (2k + 1) / 2 with the
// leading bit of 2k + 1 as the exponent.
MD_HD double int_plus_half(int k)
{
    const uint32_t v = 2u * (uint32_t)k + 1u;
#if defined(__CUDA_ARCH__)
    const int top = 31 - __clz((int)v);
#else
    const int top = 31 - __builtin_clz(v);
#endif
    const uint64_t frac = ((uint64_t)v << (52 - top)) & 0xfffffffffffffull;
    return bitsd(((uint64_t)(1023 + top - 1) << 52) | frac);
}

// floor(y) for 0 <= y < 2^31; negative y (and -0) give -1, y >= 2^31,
// infinity and NaN give INT32_MAX.  (The hardware's floor gives 0 for -0
// and NaN; callers clamp the result into a range that starts at 0, where
// only NaN then differs.)
MD_HD int floor_bits(double y)
{
    const uint64_t u = dbits(y);
    if (u >> 63) return -1;
    const int e = (int)(u >> 52) - 1023;
    if (e < 0) return 0;
    if (e > 30) return 0x7fffffff;
    const uint64_t m = (u & 0xfffffffffffffull) | (1ull << 52);
    return (int)(m >> (52 - e));
}

}  // namespace mdk
