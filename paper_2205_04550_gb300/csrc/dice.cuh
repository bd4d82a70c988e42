// dice.cuh -- the Dice coefficient of Section 2.3 (Ezhov et al. 2022) as an
// IEEE binary64 value, 2 I / (P + E) rounded to nearest-even, computed with
// integer arithmetic.
//
// On this GPU a binary64 division costs about 640 cycles of latency and a
// 64-bit integer division about 450, so scoring with either showed up in the
// scans' tails.  For integer operands the correctly rounded quotient follows
// from long division: the numerator is first shifted to the denominator's
// bit length (quotient in [1/2, 1)), the next 54 quotient bits are found as
// three digits of 18 bits, and the top 53 are rounded to nearest-even with
// the 54th as the round bit and a non-zero remainder as the sticky bit.  Each
// digit is estimated from a binary32 reciprocal of the denominator -- the
// estimate is within 1/16 of the exact quotient of the partial remainder,
// which is below 2^18, since every binary32 operation adds at most 2^-24
// relative error -- and corrected by at most one from the exact 64-bit
// remainder, so the digits are exact.  The same code compiles for the host,
// where the tests compare it with the host's IEEE division.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define DBQ_HD __host__ __device__ __forceinline__
#else
#define DBQ_HD inline
#endif

namespace dbq {

DBQ_HD int clz32(uint32_t x)
{
#if defined(__CUDA_ARCH__)
    return __clz(x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

DBQ_HD float recip_f32(uint32_t den)
{
#if defined(__CUDA_ARCH__)
    return __frcp_rn(__uint2float_rn(den));
#else
    return 1.0f / (float)den;
#endif
}

DBQ_HD uint32_t digit_estimate(uint32_t x, float r18)
{
#if defined(__CUDA_ARCH__)
    return __float2uint_rz(__fmul_rn(__uint2float_rn(x), r18));
#else
    return (uint32_t)((float)x * r18);
#endif
}

// Bits of the binary64 nearest to num / den (ties to even), 0 < num < den.
DBQ_HD uint64_t quotient_bits(uint32_t num, uint32_t den)
{
    int sh = clz32(num) - clz32(den);          // num << sh has den's bit length
    uint32_t a = num << sh;
    if (a >= den) {                            // then sh >= 1, and a / den in [1/2, 1)
        --sh;
        a >>= 1;
    }
    // q = floor(a * 2^54 / den), in [2^53, 2^54), three digits of 18 bits;
    // x is the partial remainder, below den
    const float r18 = recip_f32(den) * 262144.0f;        // 2^18 / den, scaled exactly
    uint64_t q = 0;
    uint32_t x = a;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int64_t digit = (int64_t)digit_estimate(x, r18);
        int64_t rem = ((int64_t)x << 18) - digit * (int64_t)den;
        if (rem < 0) {
            --digit;
            rem += den;
        } else if (rem >= (int64_t)den) {
            ++digit;
            rem -= den;
        }
        q = (q << 18) | (uint64_t)digit;
        x = (uint32_t)rem;
    }
    uint64_t m = q >> 1;                       // 53 bits, leading bit 52
    const bool round = q & 1u;
    const bool sticky = x != 0u;
    int e = -1 - sh;                           // num / den = m * 2^(e - 52), m in [2^52, 2^53)
    if (round && (sticky || (m & 1u))) ++m;
    if (m >> 53) {                             // rounded up to the next power of two
        m >>= 1;
        ++e;
    }
    return ((uint64_t)(e + 1023) << 52) | (m & ((1ull << 52) - 1));
}

// Dice = 2 I / (P + E) in binary64, round to nearest-even; both masks empty
// gives 1 (the reading taken for an empty pair).  Counts come from masks, so
// 2 I <= P + E < 2^32.
DBQ_HD uint64_t dice_bits(uint32_t inter, uint32_t a, uint32_t b)
{
    const uint32_t den = a + b;
    const uint32_t num = 2u * inter;
    if (den == 0u || num == den) return 0x3FF0000000000000ull;   // 1.0
    if (num == 0u) return 0;                                      // +0.0
    return quotient_bits(num, den);
}

DBQ_HD double bits_to_double(uint64_t u)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double d;
    std::memcpy(&d, &u, sizeof d);
    return d;
#endif
}

}  // namespace dbq
