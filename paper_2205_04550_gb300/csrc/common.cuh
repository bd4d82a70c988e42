// common.cuh -- device helpers shared by the query kernels of libdbq.
//
// Ranking (Section 2.3 of Ezhov et al. 2022: the entry with the largest
// combined Dice is the best match): a candidate is (score, index, payload)
// and the order is score descending, then index ascending, so the result
// does not depend on how CTAs were scheduled.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dice.cuh"

namespace dbq {

// Ranking keys are unsigned 64-bit integers whose order is the ranking order:
// a non-negative binary64 score's bit pattern (Dice scores are >= 0), or the
// complement of a non-negative binary32 distance's bit pattern (smaller
// distance = larger key).  Integer compares keep the top-k off the slow
// FP64 pipe.  The sentinel key 0 with the largest index loses to everything.
constexpr uint64_t kSentinelKey = 0ull;
constexpr int64_t kSentinelIndex = INT64_MAX;

// Device-side copy of dbq_hit (same layout as the C ABI struct).
struct Hit {
    int64_t index;
    double score;
    uint32_t i1, i2, e1, e2, p1, p2;
};
static_assert(sizeof(Hit) == 40, "Hit must match dbq_hit");

// One candidate of a per-CTA list; pay0/pay1 carry the entry's counts.
struct Cand {
    uint64_t key;
    int64_t index;
    uint64_t pay0;
    uint64_t pay1;
};

__device__ __forceinline__ bool better(uint64_t ka, int64_t ia, uint64_t kb, int64_t ib)
{
    return ka > kb || (ka == kb && ia < ib);
}

__device__ __forceinline__ uint64_t score_key(double score)   // score >= 0
{
    return (uint64_t)__double_as_longlong(score);
}

__device__ __forceinline__ double key_score(uint64_t key)
{
    return __longlong_as_double((long long)key);
}

__device__ __forceinline__ uint64_t distance_key(float d)      // d >= 0
{
    return (uint64_t)(~__float_as_uint(d));
}

// Streaming 128-bit load: read-only path, no L1 allocation, 256-byte L2
// prefetch -- the database is read once per query.
__device__ __forceinline__ uint4 ld_stream(const uint4* p)
{
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ uint32_t popc_and4(const uint4& a, const uint4& b)
{
    return __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
}

// Dice from exact counts, IEEE binary64 round-to-nearest; both empty -> 1
// (integer arithmetic, see dice.cuh).
__device__ __forceinline__ double dice_rn(uint32_t inter, uint32_t a, uint32_t b)
{
    return bits_to_double(dice_bits(inter, a, b));
}

__device__ __forceinline__ double score_rn(uint32_t i1, uint32_t i2, uint32_t e1, uint32_t e2,
                                           uint32_t p1, uint32_t p2)
{
    return __dmul_rn(__dadd_rn(dice_rn(i1, p1, e1), dice_rn(i2, p2, e2)), 0.5);
}

__host__ __device__ __forceinline__ int next_pow2(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace dbq
