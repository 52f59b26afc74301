// div_small.cuh -- correctly rounded s / N for the centre of Eq. 2, with one
// FP64 multiplication and integer arithmetic.
//
// q0 = RN(s * y) with y = RN(1/N) lies within two units in the last place of
// s/N (relative error below 2^-52 against a unit of at least 2^-53 q0).  The
// remainder of q0 is exact in integers: with s = Ms 2^Es and q0 = Mq 2^Eq
// (53-bit significands, Es > Eq),
//   s - q0 N = (Ms 2^(Es - Eq) - Mq N) 2^Eq = r 2^Eq,
// so s/N = (Mq + r/N) 2^Eq and the rounded quotient is Mq + k with k the
// integer nearest to r/N, |k| <= 2.  Adding k to
// the bit pattern of q0 steps through the representable values, also onto
// the top of the binade (Mq + k = 2^53).  Where Mq + k leaves [2^52, 2^53]
// the candidates are spaced differently; that case, and operands where
// anything could under- or overflow, take the IEEE division.
//
// Compiles for the host too, so the CPU tests run this code against the
// host's IEEE division.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define SLS_DS_HD __host__ __device__ __forceinline__
#else
#define SLS_DS_HD static inline
#endif

namespace sls {
namespace divs {

SLS_DS_HD uint64_t bits_of(double v)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(v);
#else
    uint64_t b;
    memcpy(&b, &v, sizeof b);
    return b;
#endif
}

SLS_DS_HD double of_bits(uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double v;
    memcpy(&v, &b, sizeof v);
    return v;
#endif
}

SLS_DS_HD double mul_rn(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}

SLS_DS_HD double div_rn(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __ddiv_rn(a, b);
#else
    return a / b;
#endif
}

// RN(s / N) for an integer 2 <= N <= 16, given y = RN(1/N) and fN = N as a
// double.  Returns the quotient's bit pattern.
SLS_DS_HD uint64_t div_small_bits(uint64_t sb, uint32_t N, double y, double fN)
{
    const uint32_t es = (uint32_t)(sb >> 52) & 0x7ffu;
    // normal s well inside the range: q0 and the quotient are normal too
    if (es - 63u > 1937u) return bits_of(div_rn(of_bits(sb), fN));
    const uint64_t qb = bits_of(mul_rn(of_bits(sb), y));
    const uint32_t eq = (uint32_t)(qb >> 52) & 0x7ffu;
    const uint64_t ms = (sb & 0x000fffffffffffffull) | 0x0010000000000000ull;
    const uint64_t mq = (qb & 0x000fffffffffffffull) | 0x0010000000000000ull;
    // s/N < s, so eq <= es; s/N >= s/16, so es - eq <= 5
    const uint32_t de = es - eq;
    const int64_t r = (int64_t)(ms << de) - (int64_t)(mq * N);
    // |r/N| against 1/2 and 3/2.  A quotient of two doubles is never exactly
    // halfway between two doubles (s = N (2M + 1) 2^(E-1) would need more than
    // 53 significant bits), so no tie can occur.
    const int64_t n = (int64_t)N, a2 = r < 0 ? -2 * r : 2 * r;
    if (a2 > 5 * n) return bits_of(div_rn(of_bits(sb), fN));
    int64_t k = (int64_t)(a2 > n) + (int64_t)(a2 > 3 * n);
    if (r < 0) k = -k;
    const int64_t mk = (int64_t)mq + k;
    if (mk < (int64_t)0x0010000000000000ll || mk > (int64_t)0x0020000000000000ll)
        return bits_of(div_rn(of_bits(sb), fN));
    return qb + (uint64_t)k;
}

}  // namespace divs
}  // namespace sls
