// topk.cuh -- block-level running top-k and the cross-CTA merge used by the
// fused query kernels.
//
// The best match of Section 2.3 (Ezhov et al. 2022) is the entry with the
// largest combined Dice; the top-k generalises it.  Order: score
// descending, then database index ascending, so the result is independent of
// CTA scheduling.  Candidates carry two 64-bit payload words (the entry's
// counts) so the final hits need no second pass over the database.
//
// Shared-memory protocol (all threads of the block take part in every call):
//   * slots [0, k) hold the running top-k, best first, padded with sentinels;
//   * topk_offer() appends a candidate at k + (atomic counter) when it beats
//     the current k-th best -- at most kTopkCap - k offers between flushes;
//   * topk_flush() bitonic-sorts the k + appended slots and keeps the first k.
// After the scan each CTA publishes its k slots to global scratch and the
// last CTA to arrive (atomicInc ticket that wraps to zero, no spinning)
// merges all of them with the same offer/flush rounds.
#pragma once

#include "common.cuh"

namespace dbq {

constexpr int kTopkCap = 2048;

struct TopK {
    uint64_t* key;    // [kTopkCap] ranking keys (see common.cuh)
    int64_t* idx;     // [kTopkCap]
    uint64_t* pay0;   // [kTopkCap]
    uint64_t* pay1;   // [kTopkCap]
    int* misc;        // [0] appended count, [1] is-last flag
};

constexpr size_t topk_smem_bytes() { return (size_t)kTopkCap * 32 + 4 * sizeof(int); }

// Carve a TopK from `p` (8-byte aligned); returns the first byte after it.
__device__ __forceinline__ unsigned char* topk_carve(TopK& t, unsigned char* p)
{
    t.key = reinterpret_cast<uint64_t*>(p);
    p += kTopkCap * sizeof(uint64_t);
    t.idx = reinterpret_cast<int64_t*>(p);
    p += kTopkCap * sizeof(int64_t);
    t.pay0 = reinterpret_cast<uint64_t*>(p);
    p += kTopkCap * sizeof(uint64_t);
    t.pay1 = reinterpret_cast<uint64_t*>(p);
    p += kTopkCap * sizeof(uint64_t);
    t.misc = reinterpret_cast<int*>(p);
    p += 4 * sizeof(int);
    return p;
}

__device__ __forceinline__ void topk_clear_slot(TopK& t, int i)
{
    t.key[i] = kSentinelKey;
    t.idx[i] = kSentinelIndex;
    t.pay0[i] = 0;
    t.pay1[i] = 0;
}

// Sentinels everywhere; call before first use.  Ends with a barrier.
__device__ __forceinline__ void topk_init(TopK& t)
{
    for (int i = threadIdx.x; i < kTopkCap; i += blockDim.x) topk_clear_slot(t, i);
    if (threadIdx.x == 0) t.misc[0] = 0;
    __syncthreads();
}

__device__ __forceinline__ void topk_offer(TopK& t, int k, uint64_t key, int64_t index,
                                           uint64_t p0, uint64_t p1)
{
    if (better(key, index, t.key[k - 1], t.idx[k - 1])) {
        const int pos = k + atomicAdd(&t.misc[0], 1);
        t.key[pos] = key;
        t.idx[pos] = index;
        t.pay0[pos] = p0;
        t.pay1[pos] = p1;
    }
}

// Binary32 Dice: 2 I / (P + E) with both operands and the quotient rounded
// to nearest, each within a relative 2^-24 of exact; both empty -> 1.
__device__ __forceinline__ float dice_f32(uint32_t inter, uint32_t a, uint32_t b)
{
    const uint32_t den = a + b;
    if (den == 0u) return 1.0f;
    return __fdiv_rn((float)(2u * inter), (float)den);
}

// Offer an entry by its counts.  The binary64 score (the ranking key) costs
// two binary64 divisions, which are slow on this GPU; most entries of a scan
// cannot reach the current k-th best, and a binary32 bound shows it first:
// each binary32 Dice is within a relative 3 x 2^-24 of the exact quotient and
// their sum within one more 2^-24, so the score times (1 + 2^-20) is an upper
// bound of the exact score and of its binary64 rounding.  An entry whose bound
// is below the k-th best score is strictly worse than it (no tie is possible)
// and is skipped; every other entry is scored exactly and offered as before,
// so the result is the same.
__device__ __forceinline__ void topk_offer_counts(TopK& t, int k, uint32_t i1, uint32_t i2,
                                                  uint32_t e1, uint32_t e2, uint32_t p1,
                                                  uint32_t p2, int64_t index)
{
    const uint64_t kth = t.key[k - 1];
    if (kth != kSentinelKey) {
        const float up = (dice_f32(i1, p1, e1) + dice_f32(i2, p2, e2)) * (0.5f + 0x1p-21f);
        if ((double)up < key_score(kth)) return;
    }
    topk_offer(t, k, score_key(score_rn(i1, i2, e1, e2, p1, p2)), index,
               (uint64_t)i1 | ((uint64_t)i2 << 32), (uint64_t)e1 | ((uint64_t)e2 << 32));
}

__device__ __forceinline__ void bitonic_sort_topk(TopK& t, int n)
{
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const bool hi_better = better(t.key[hi], t.idx[hi], t.key[lo], t.idx[lo]);
                if (hi_better == up) {
                    const uint64_t kk = t.key[lo]; t.key[lo] = t.key[hi]; t.key[hi] = kk;
                    const int64_t ii = t.idx[lo]; t.idx[lo] = t.idx[hi]; t.idx[hi] = ii;
                    const uint64_t a = t.pay0[lo]; t.pay0[lo] = t.pay0[hi]; t.pay0[hi] = a;
                    const uint64_t b = t.pay1[lo]; t.pay1[lo] = t.pay1[hi]; t.pay1[hi] = b;
                }
            }
            __syncthreads();
        }
    }
}

// Merge the appended candidates into slots [0, k).  Starts and ends with a
// barrier.  A round of at most kRankFlush appended candidates (the common
// case once the k best are established, and in small scans) is merged by
// counting every element's new position directly -- its rank among the
// sorted k (a binary search, or its own slot) plus the appended candidates
// better than it -- and writing it there: three barriers, where a bitonic
// sort of the same elements takes one per stage (15 for 32 elements), and the
// barriers of a 1024-thread block are the expensive part.  Larger rounds use
// the bitonic sort, whose cost does not grow with the round as fast as the
// direct count does.
constexpr int kRankFlush = 64;

__device__ __forceinline__ void topk_flush(TopK& t, int k)
{
    __syncthreads();
    const int added = t.misc[0];
    if (added > 0) {
        const int n = k + added;
        if (added <= kRankFlush && n <= (int)blockDim.x) {
            const int i = threadIdx.x;
            uint64_t ki = 0, p0 = 0, p1 = 0;
            int64_t ii = kSentinelIndex;
            int rank = k;
            if (i < n) {
                ki = t.key[i];
                ii = t.idx[i];
                p0 = t.pay0[i];
                p1 = t.pay1[i];
                if (ii != kSentinelIndex) {
                    int r;
                    if (i < k) {
                        r = i;                      // the sorted slots before it are better
                    } else {                        // sorted slots better than it
                        int lo = 0, hi = k;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (better(t.key[mid], t.idx[mid], ki, ii)) lo = mid + 1;
                            else hi = mid;
                        }
                        r = lo;
                    }
                    // appended candidates better than it (itself is not)
                    int j = k;
                    for (; j + 8 <= n; j += 8) {
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            r += better(t.key[j + u], t.idx[j + u], ki, ii) ? 1 : 0;
                    }
                    for (; j < n; ++j) r += better(t.key[j], t.idx[j], ki, ii) ? 1 : 0;
                    rank = r;
                }
            }
            __syncthreads();   // every element read before any is moved
            if (i < n) {
                // ranks are distinct and below k, so no move lands in [k, n),
                // which is cleared; slots of [0, k) left unwritten already hold
                // sentinels (the k best never shrink)
                if (rank < k) {
                    t.key[rank] = ki;
                    t.idx[rank] = ii;
                    t.pay0[rank] = p0;
                    t.pay1[rank] = p1;
                }
                if (i >= k) topk_clear_slot(t, i);
            }
        } else {
            const int n2 = next_pow2(n);
            bitonic_sort_topk(t, n2);
            for (int i = k + threadIdx.x; i < n2; i += blockDim.x) topk_clear_slot(t, i);
        }
    }
    if (threadIdx.x == 0) t.misc[0] = 0;
    __syncthreads();
}

// Publish the k slots to dst[slot * k ...] and take a ticket on a counter
// shared by `nslots` publishers.  Returns true (in every thread) in the last
// publisher to arrive, which then sees every list.
__device__ __forceinline__ bool topk_publish_slot(TopK& t, int k, Cand* dst, int slot, int nslots,
                                                  unsigned int* ticket)
{
    Cand* mine = dst + (int64_t)slot * k;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        Cand c;
        c.key = t.key[j];
        c.index = t.idx[j];
        c.pay0 = t.pay0[j];
        c.pay1 = t.pay1[j];
        mine[j] = c;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int done = atomicInc(ticket, (unsigned int)nslots - 1);   // wraps to 0
        t.misc[1] = (done == (unsigned int)nslots - 1) ? 1 : 0;
    }
    __syncthreads();
    const bool last = t.misc[1] != 0;
    if (last) __threadfence();
    return last;
}

// One slot per CTA of the grid.
__device__ __forceinline__ bool topk_publish(TopK& t, int k, Cand* cand, unsigned int* ticket)
{
    return topk_publish_slot(t, k, cand, blockIdx.x, gridDim.x, ticket);
}

// Merge of m / k published lists, each sorted best first (every list comes
// from a flushed or merged TopK), when they fit in half of the shared slots:
// every candidate's final position is its position in its own list plus the
// number of candidates of each other list that are better (a binary search
// per list), and the first k positions are written to the upper half of the
// slots, then moved down to [0, k).  The order is strict (entry indices are
// unique), so positions never collide; sentinels are never better than a
// real candidate and are not placed.
// Up to 32 sorted lists of at most kTournamentK candidates are merged by one
// warp: lane l holds the current head of list l, and each round a butterfly
// of shuffles finds the best head in every lane, whose lane writes it out and
// advances.  k rounds of a few dozen instructions, where ranking every
// candidate by binary searches in every other list reads shared memory at
// scattered addresses (bank conflicts) and, at these sizes, takes several
// times longer.
constexpr int kTournamentK = 16;

__device__ __forceinline__ void topk_tournament(TopK& t, int k, int lists, int out0)
{
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    int pos = 0;
    uint64_t hk = kSentinelKey;
    int64_t hi = kSentinelIndex;
    if (lane < lists) {
        hk = t.key[lane * k];
        hi = t.idx[lane * k];
    }
    for (int r = 0; r < k; ++r) {
        uint64_t bk = hk;
        int64_t bi = hi;
        int bl = lane;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const uint64_t ok = __shfl_xor_sync(0xffffffffu, bk, off);
            const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, off);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, off);
            if (better(ok, oi, bk, bi)) {
                bk = ok;
                bi = oi;
                bl = ol;
            }
        }
        if (bi == kSentinelIndex) break;               // every list exhausted
        if (lane == bl) {
            const int j = lane * k + pos;
            t.key[out0 + r] = hk;
            t.idx[out0 + r] = hi;
            t.pay0[out0 + r] = t.pay0[j];
            t.pay1[out0 + r] = t.pay1[j];
            ++pos;
            if (pos < k) {
                hk = t.key[j + 1];
                hi = t.idx[j + 1];
            } else {
                hk = kSentinelKey;
                hi = kSentinelIndex;
            }
        }
    }
}

__device__ __forceinline__ bool topk_merge_sorted(TopK& t, int k, const Cand* cand, int64_t m)
{
    constexpr int kHalf = kTopkCap / 2;
    if (m % k != 0 || m > kHalf || k > kHalf) return false;
    const int lists = (int)(m / k);
    if (k <= kTournamentK && lists <= 32) {
        for (int i = threadIdx.x; i < kTopkCap; i += blockDim.x) {
            if (i < (int)m) {
                const Cand* src = cand + i;
                t.key[i] = __ldcg(reinterpret_cast<const unsigned long long*>(&src->key));
                t.idx[i] = __ldcg(reinterpret_cast<const long long*>(&src->index));
                t.pay0[i] = __ldcg(reinterpret_cast<const unsigned long long*>(&src->pay0));
                t.pay1[i] = __ldcg(reinterpret_cast<const unsigned long long*>(&src->pay1));
            } else {
                topk_clear_slot(t, i);
            }
        }
        __syncthreads();
        topk_tournament(t, k, lists, kHalf);
        __syncthreads();
        for (int i = threadIdx.x; i < k; i += blockDim.x) {   // [kHalf, kHalf + k) -> [0, k)
            t.key[i] = t.key[kHalf + i];
            t.idx[i] = t.idx[kHalf + i];
            t.pay0[i] = t.pay0[kHalf + i];
            t.pay1[i] = t.pay1[kHalf + i];
        }
        __syncthreads();
        for (int i = k + threadIdx.x; i < kTopkCap; i += blockDim.x) topk_clear_slot(t, i);
        if (threadIdx.x == 0) t.misc[0] = 0;
        __syncthreads();
        return true;
    }
    for (int i = threadIdx.x; i < kTopkCap; i += blockDim.x) {
        if (i < (int)m) {
            const Cand* src = cand + i;
            t.key[i] = __ldcg(reinterpret_cast<const unsigned long long*>(&src->key));
            t.idx[i] = __ldcg(reinterpret_cast<const long long*>(&src->index));
            t.pay0[i] = __ldcg(reinterpret_cast<const unsigned long long*>(&src->pay0));
            t.pay1[i] = __ldcg(reinterpret_cast<const unsigned long long*>(&src->pay1));
        } else if (i >= kHalf) {
            topk_clear_slot(t, i);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (int)m; i += blockDim.x) {
        const uint64_t ck = t.key[i];
        const int64_t ci = t.idx[i];
        if (ci == kSentinelIndex) continue;
        const int own = i / k;
        int r = i - own * k;
        for (int l = 0; l < lists && r < k; ++l) {
            if (l == own) continue;
            // the candidates of list l better than this one form a prefix
            int lo = 0, hi = k;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                const int j = l * k + mid;
                if (better(t.key[j], t.idx[j], ck, ci)) lo = mid + 1;
                else hi = mid;
            }
            r += lo;
        }
        if (r < k) {
            t.key[kHalf + r] = ck;
            t.idx[kHalf + r] = ci;
            t.pay0[kHalf + r] = t.pay0[i];
            t.pay1[kHalf + r] = t.pay1[i];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHalf; i += blockDim.x) {
        if (i < k) {
            t.key[i] = t.key[kHalf + i];
            t.idx[i] = t.idx[kHalf + i];
            t.pay0[i] = t.pay0[kHalf + i];
            t.pay1[i] = t.pay1[kHalf + i];
        } else {
            topk_clear_slot(t, i);
        }
    }
    __syncthreads();
    for (int i = kHalf + threadIdx.x; i < kTopkCap; i += blockDim.x) topk_clear_slot(t, i);
    if (threadIdx.x == 0) t.misc[0] = 0;
    __syncthreads();
    return true;
}

// In the last CTA: merge the m published candidates into slots [0, k).
__device__ __forceinline__ void topk_merge_published(TopK& t, int k, const Cand* cand, int64_t m)
{
    if (topk_merge_sorted(t, k, cand, m)) return;
    for (int i = threadIdx.x; i < kTopkCap; i += blockDim.x) topk_clear_slot(t, i);
    if (threadIdx.x == 0) t.misc[0] = 0;
    __syncthreads();
    const int round = kTopkCap - k;
    for (int64_t r0 = 0; r0 < m; r0 += round) {
        for (int j = threadIdx.x; j < round; j += blockDim.x) {
            const int64_t r = r0 + j;
            if (r < m) {
                const Cand* src = cand + r;
                const unsigned long long sc =
                    __ldcg(reinterpret_cast<const unsigned long long*>(&src->key));
                const long long ix = __ldcg(reinterpret_cast<const long long*>(&src->index));
                if (ix != kSentinelIndex) {
                    const unsigned long long p0 =
                        __ldcg(reinterpret_cast<const unsigned long long*>(&src->pay0));
                    const unsigned long long p1 =
                        __ldcg(reinterpret_cast<const unsigned long long*>(&src->pay1));
                    topk_offer(t, k, (uint64_t)sc, (int64_t)ix, (uint64_t)p0, (uint64_t)p1);
                }
            }
        }
        topk_flush(t, k);
    }
}

constexpr int kMergeGroup = 16;  // CTAs per first-level merge group

// Two-level publication for a grid of CTAs: every CTA publishes its list to
// cand[blockIdx.x * k]; the last CTA to finish in each group of kMergeGroup
// merges its group's lists into group_lists[group * k] (while other CTAs may
// still be scanning), and the last group merger merges the group lists.
// tickets[0] is the top-level counter, tickets[1 + g] group g's (all zero
// between launches).  Returns true, in every thread, in the CTA that then
// holds the final list in slots [0, k).
__device__ __forceinline__ bool topk_publish_two_level(TopK& t, int k, Cand* cand,
                                                       Cand* group_lists, unsigned int* tickets)
{
    const int group = blockIdx.x / kMergeGroup;
    const int first = group * kMergeGroup;
    const int members = min(kMergeGroup, (int)gridDim.x - first);
    const int ngroups = ((int)gridDim.x + kMergeGroup - 1) / kMergeGroup;
    if (!topk_publish_slot(t, k, cand + (int64_t)first * k, blockIdx.x - first, members,
                           tickets + 1 + group))
        return false;
    topk_merge_published(t, k, cand + (int64_t)first * k, (int64_t)members * k);
    if (!topk_publish_slot(t, k, group_lists, group, ngroups, tickets))
        return false;
    topk_merge_published(t, k, group_lists, (int64_t)ngroups * k);
    return true;
}

}  // namespace dbq
