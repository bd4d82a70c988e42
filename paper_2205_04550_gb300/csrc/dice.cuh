// dice.cuh -- the Dice coefficient of Section 2.3 (Ezhov et al. 2022) as an
// IEEE binary64 value, 2 I / (P + E) rounded to nearest-even, computed with
// integer arithmetic.
//
// On this GPU a binary64 division costs about 640 cycles of latency and the
// binary64 pipe is narrow, so scoring every entry of a scan with __ddiv_rn
// showed up in the scans' tails.  For integer operands the correctly rounded
// quotient follows from two 64-bit integer divisions: the numerator is first
// shifted to the denominator's bit length (quotient in [1/2, 1)), the next 64
// quotient bits are taken as floor(num * 2^64 / den) in two 32-bit steps, and
// the top 53 of them are rounded to nearest-even with the 54th bit as the
// round bit and everything below it, remainder included, as the sticky bit.
// The header compiles for the host as well, where the tests compare it with
// the host's IEEE division.
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

// Bits of the binary64 nearest to num / den (ties to even), 0 < num < den.
DBQ_HD uint64_t quotient_bits(uint32_t num, uint32_t den)
{
    int sh = clz32(num) - clz32(den);          // num << sh has den's bit length
    uint32_t a = num << sh;
    if (a >= den) {                            // then sh >= 1, and a / den in [1/2, 1)
        --sh;
        a >>= 1;
    }
    const uint64_t a1 = (uint64_t)a << 32;
    const uint64_t q1 = a1 / den;              // in [2^31, 2^32)
    const uint64_t r1 = a1 - q1 * den;
    const uint64_t a2 = r1 << 32;
    const uint64_t q2 = a2 / den;              // below 2^32
    const uint64_t r2 = a2 - q2 * den;
    const uint64_t q = (q1 << 32) | q2;        // floor(a * 2^64 / den), in [2^63, 2^64)
    uint64_t m = q >> 11;                      // 53 bits, leading bit 52
    const bool round = (q >> 10) & 1u;
    const bool sticky = (q & 0x3FFu) != 0 || r2 != 0;
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
