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
// barrier.  When the k slots and the appended candidates fit in one element
// per thread, every element's new position is counted directly -- its rank
// among the sorted k (a binary search, or its own slot) plus the appended
// candidates better than it -- and written in one step: three barriers in all,
// where a bitonic sort of the same elements takes one per stage (15 for 32
// elements, 45 for 512), and a barrier of a 1024-thread block is the
// expensive part here.  Larger rounds use the bitonic sort.
__device__ __forceinline__ void topk_flush(TopK& t, int k)
{
    __syncthreads();
    const int added = t.misc[0];
    if (added > 0) {
        const int n = k + added;
        if (n <= (int)blockDim.x) {
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
                    for (int j = k; j < n && r < k; ++j)      // appended candidates better than it
                        if (j != i && better(t.key[j], t.idx[j], ki, ii)) ++r;
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
// from a flushed or merged TopK), when they fit in the shared slots with
// room for k more and one entry per warp.  The k-th element of every list
// bounds the answer: the list with the best k-th element alone holds k
// candidates at least that good, so no candidate worse than T (the best of
// the k-th elements) can be among the k best.  The few candidates at least
// as good as T are ranked exactly -- a candidate's final position is the
// number of candidates better than it, summed over the lists by binary
// searches that the 32 lanes of a warp share -- and written at that
// position.  The order is strict (entry indices are unique), so positions
// never collide; sentinels are never better than a real candidate and are not
// placed.  Five barriers, whatever the number of lists.
__device__ __forceinline__ bool topk_merge_sorted(TopK& t, int k, const Cand* cand, int64_t m)
{
    const int nwarps = (int)(blockDim.x >> 5);
    if (m % k != 0 || m + k + nwarps > kTopkCap) return false;
    const int mm = (int)m;
    const int lists = mm / k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kTopkCap; i += blockDim.x) {
        if (i < mm) {
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
    // T: the best k-th element over the lists (block reduction)
    uint64_t tk = kSentinelKey;
    int64_t ti = kSentinelIndex;
    for (int l = threadIdx.x; l < lists; l += blockDim.x) {
        const int j = l * k + k - 1;
        if (better(t.key[j], t.idx[j], tk, ti)) {
            tk = t.key[j];
            ti = t.idx[j];
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const uint64_t ok = __shfl_down_sync(0xffffffffu, tk, off);
        const int64_t oi = __shfl_down_sync(0xffffffffu, ti, off);
        if (better(ok, oi, tk, ti)) {
            tk = ok;
            ti = oi;
        }
    }
    if (lane == 0) {
        t.key[mm + k + warp] = tk;
        t.idx[mm + k + warp] = ti;
    }
    __syncthreads();
    tk = kSentinelKey;
    ti = kSentinelIndex;
    for (int w = 0; w < nwarps; ++w)
        if (better(t.key[mm + k + w], t.idx[mm + k + w], tk, ti)) {
            tk = t.key[mm + k + w];
            ti = t.idx[mm + k + w];
        }
    // every candidate not worse than T: its exact rank, by one warp
    for (int base = warp * 32; base < mm; base += (int)blockDim.x) {
        const int i = base + lane;
        uint64_t ck = 0;
        int64_t ci = kSentinelIndex;
        if (i < mm) {
            ck = t.key[i];
            ci = t.idx[i];
        }
        const bool keep = ci != kSentinelIndex && !better(tk, ti, ck, ci);
        unsigned int todo = __ballot_sync(0xffffffffu, keep);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint64_t xk = __shfl_sync(0xffffffffu, ck, src);
            const int64_t xi = __shfl_sync(0xffffffffu, ci, src);
            int r = 0;
            for (int l = lane; l < lists; l += 32) {    // candidates of list l better than x
                int lo = 0, hi = k;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    const int j = l * k + mid;
                    if (better(t.key[j], t.idx[j], xk, xi)) lo = mid + 1;
                    else hi = mid;
                }
                r += lo;
            }
            r = __reduce_add_sync(0xffffffffu, r);
            if (lane == src && r < k) {
                t.key[mm + r] = ck;
                t.idx[mm + r] = ci;
                t.pay0[mm + r] = t.pay0[i];
                t.pay1[mm + r] = t.pay1[i];
            }
        }
    }
    __syncthreads();
    // move [m, m + k) to [0, k) (m >= k: the ranges do not overlap), then
    // clear everything after the k slots
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        t.key[i] = t.key[mm + i];
        t.idx[i] = t.idx[mm + i];
        t.pay0[i] = t.pay0[mm + i];
        t.pay1[i] = t.pay1[mm + i];
    }
    __syncthreads();
    for (int i = k + threadIdx.x; i < kTopkCap; i += blockDim.x) topk_clear_slot(t, i);
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
