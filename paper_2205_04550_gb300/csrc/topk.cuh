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
//   * topk_offer() appends a candidate at k + (a warp's share of an atomic
//     counter) when it beats the current k-th best -- at most kTopkCap - k
//     offers between flushes;
//   * topk_flush() merges the appended candidates into the k best: by
//     direct counts for small rounds, by a merge tree (k <= kTreeK) or a
//     bitonic sort for large ones.
// After the scan each CTA publishes its k slots to global scratch and the
// last CTA to arrive (atomicInc ticket that wraps to zero, no spinning)
// merges all of them (topk_merge_published: warp tournaments, merge trees or
// ranks, else offer/flush rounds), directly or through groups of CTAs.
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

// The offering lanes of a warp that are converged here take their slots with
// one shared-memory atomic (a ballot and a prefix count), not one each: in a
// round where most candidates pass (the first group of a scan) hundreds of
// same-address atomics otherwise serialise.
__device__ __forceinline__ void topk_offer(TopK& t, int k, uint64_t key, int64_t index,
                                           uint64_t p0, uint64_t p1)
{
    const bool pass = better(key, index, t.key[k - 1], t.idx[k - 1]);
    const unsigned act = __activemask();
    const unsigned want = __ballot_sync(act, pass);
    if (want == 0u) return;
    const int lane = (int)(threadIdx.x & 31);
    const int leader = __ffs(want) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&t.misc[0], __popc(want));
    base = __shfl_sync(act, base, leader);
    if (pass) {
        const int pos = k + base + __popc(want & ((1u << lane) - 1u));
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
    bool maybe = true;
    if (kth != kSentinelKey) {
        const float up = (dice_f32(i1, p1, e1) + dice_f32(i2, p2, e2)) * (0.5f + 0x1p-21f);
        maybe = !((double)up < key_score(kth));
    }
    uint64_t key = kSentinelKey;                // a sentinel is never offered
    int64_t idx = kSentinelIndex;
    if (maybe) {
        key = score_key(score_rn(i1, i2, e1, e2, p1, p2));
        idx = index;
    }
    topk_offer(t, k, key, idx, (uint64_t)i1 | ((uint64_t)i2 << 32),
               (uint64_t)e1 | ((uint64_t)e2 << 32));
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

// Merge trees for k <= kTreeK.  A sorted list is merged with its neighbour
// by ranks: an element's position in the merged list is its position in its
// own list plus the number of elements of the other list before it, found by
// one binary search.  Ties (only sentinels compare equal) go to the left
// list, so the positions of a pair are a permutation of [0, LA + LB) and every
// output slot is written exactly once: no clearing between levels, one
// barrier per level, and log2(lists) levels of one search each, where ranking
// against every other list at once costs lists - 1 searches per element (and
// a bitonic sort one barrier per stage).  Appended candidates are first
// sorted in runs of 32 by the warps, in registers (shuffles, no barriers).
constexpr int kTreeK = 64;

// Sort slots [base, base + 32) best first in one warp; lanes at or past `len`
// count as sentinels and are written as sentinels.
__device__ __forceinline__ void warp_sort_run(TopK& t, int base, int len)
{
    const int lane = threadIdx.x & 31;
    uint64_t key = kSentinelKey;
    int64_t idx = kSentinelIndex;
    int src = lane;
    if (lane < len) {
        key = t.key[base + lane];
        idx = t.idx[base + lane];
    }
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint64_t ok = __shfl_xor_sync(0xffffffffu, key, stride);
            const int64_t oi = __shfl_xor_sync(0xffffffffu, idx, stride);
            const int os = __shfl_xor_sync(0xffffffffu, src, stride);
            const bool best_first = (lane & size) == 0;    // direction of this block
            const bool lower = (lane & stride) == 0;
            const bool take = (lower == best_first) ? better(ok, oi, key, idx)
                                                    : better(key, idx, ok, oi);
            if (take) {
                key = ok;
                idx = oi;
                src = os;
            }
        }
    }
    uint64_t p0 = 0, p1 = 0;
    if (src < len) {
        p0 = t.pay0[base + src];
        p1 = t.pay1[base + src];
    }
    __syncwarp();
    t.key[base + lane] = key;
    t.idx[base + lane] = idx;
    t.pay0[base + lane] = p0;
    t.pay1[base + lane] = p1;
}

// Number of the first n slots from `base` better than (key, idx), or, with
// `or_equal`, better than or equal to it (a prefix of a sorted list).
__device__ __forceinline__ int count_before(const TopK& t, int base, int n, uint64_t key,
                                            int64_t idx, bool or_equal)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const uint64_t mk = t.key[base + mid];
        bool before = mk > key;
        if (mk == key) {                        // the index decides (read only then)
            const int64_t mi = t.idx[base + mid];
            before = or_equal ? mi <= idx : mi < idx;
        }
        if (before) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Element q of the merge of list A (la slots at a) and list B (lb slots at
// b; with `b_empty`, lb sentinels that are not stored) goes to dst + its
// position, if that is below lout.  Reads only A and B; dst is disjoint.
__device__ __forceinline__ void merge_element(TopK& t, int a, int la, int b, int lb, bool b_empty,
                                              int q, int dst, int lout)
{
    const bool in_b = q >= la;
    const int pos = in_b ? q - la : q;
    int from = -1;
    uint64_t key = kSentinelKey;
    int64_t idx = kSentinelIndex;
    if (!in_b) from = a + pos;
    else if (!b_empty) from = b + pos;
    if (from >= 0) {
        key = t.key[from];
        idx = t.idx[from];
    }
    int r = pos;
    if (!in_b) {
        if (!b_empty) r += count_before(t, b, lb, key, idx, false);
    } else {
        r += b_empty ? la : count_before(t, a, la, key, idx, true);
    }
    if (r < lout) {
        t.key[dst + r] = key;
        t.idx[dst + r] = idx;
        t.pay0[dst + r] = from >= 0 ? t.pay0[from] : 0;
        t.pay1[dst + r] = from >= 0 ? t.pay1[from] : 0;
    }
}

// One level: lists i < nl of l slots at src + i * l are merged in pairs
// (2p, 2p + 1), the first lout slots of pair p going to dst + p * lout; a
// last unpaired list is merged with an empty one (copied and padded).
// Ends with a barrier.
__device__ __forceinline__ void merge_level(TopK& t, int src, int l, int nl, int dst, int lout)
{
    const int npairs = (nl + 1) >> 1;
    const int total = npairs * 2 * l;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int p = e / (2 * l);
        const int q = e - p * 2 * l;
        merge_element(t, src + 2 * p * l, l, src + (2 * p + 1) * l, l, 2 * p + 1 >= nl, q,
                      dst + p * lout, lout);
    }
    __syncthreads();
}

// Slots taken by the levels of a tree over nl lists of l slots, alternating
// between regions `a` (holding the lists) and `b`: the furthest slot written
// in each, and the region and length of the result.
struct TreeSpan {
    int end_a, end_b, res, len;
};

__device__ __forceinline__ TreeSpan tree_span(int a, int b, int l, int nl, int k)
{
    TreeSpan s{a + l * nl, b, a, l};
    int src = a, dst = b;
    while (nl > 1) {
        const int lout = min(k, 2 * l);
        nl = (nl + 1) >> 1;
        const int end = dst + nl * lout;
        if (dst == b) s.end_b = max(s.end_b, end);
        else s.end_a = max(s.end_a, end);
        l = lout;
        const int tmp = src;
        src = dst;
        dst = tmp;
    }
    s.res = src;
    s.len = l;
    return s;
}

__device__ __forceinline__ void merge_tree(TopK& t, int a, int b, int l, int nl, int k)
{
    int src = a, dst = b;
    while (nl > 1) {
        const int lout = min(k, 2 * l);
        merge_level(t, src, l, nl, dst, lout);
        nl = (nl + 1) >> 1;
        l = lout;
        const int tmp = src;
        src = dst;
        dst = tmp;
    }
}

// The merge-tree flush and the merge of published lists are not inlined:
// they run once per round or per scan, and inlined they raised the register
// pressure of the scan loops around them to the point of spilling.  They
// take the TopK by value, so its pointers stay in registers.
//
// Flush by a merge tree: the appended candidates are sorted in runs of 32,
// the runs merged pairwise, alternating between their own slots and the
// slots after them, and the result merged with [0, k).  Returns false, having done
// nothing, when the levels do not fit the slots.  Slots past k are left
// holding sentinels.
static __device__ __noinline__ bool topk_flush_tree(TopK t, int k, int added)
{
    const int runs = (added + 31) >> 5;
    const int b = k + 32 * runs;                         // scratch region after the runs
    const TreeSpan sp = tree_span(k, b, 32, runs, k);
    const int fin = sp.res == k ? b : k;                 // the region not holding the runs' result
    const int end_a = max(sp.end_a, fin == k ? 2 * k : 0);
    const int end_b = max(sp.end_b, fin == b ? b + k : 0);
    if (end_a > b || end_b > kTopkCap) return false;
    const int warp = (int)(threadIdx.x >> 5);
    const int warps = (int)(blockDim.x >> 5);
    for (int r = warp; r < runs; r += warps) warp_sort_run(t, k + 32 * r, min(32, added - 32 * r));
    __syncthreads();
    merge_tree(t, k, b, 32, runs, k);
    for (int q = threadIdx.x; q < k + sp.len; q += blockDim.x)
        merge_element(t, 0, k, sp.res, sp.len, false, q, fin, k);
    __syncthreads();
    uint64_t ck = 0, cp0 = 0, cp1 = 0;
    int64_t ci = 0;
    const bool mover = (int)threadIdx.x < k;
    if (mover) {
        ck = t.key[fin + threadIdx.x];
        ci = t.idx[fin + threadIdx.x];
        cp0 = t.pay0[fin + threadIdx.x];
        cp1 = t.pay1[fin + threadIdx.x];
    }
    __syncthreads();
    if (mover) {
        t.key[threadIdx.x] = ck;
        t.idx[threadIdx.x] = ci;
        t.pay0[threadIdx.x] = cp0;
        t.pay1[threadIdx.x] = cp1;
    }
    for (int i = k + threadIdx.x; i < end_a; i += blockDim.x) topk_clear_slot(t, i);
    for (int i = b + threadIdx.x; i < end_b; i += blockDim.x) topk_clear_slot(t, i);
    return true;
}

// Merge the appended candidates into slots [0, k).  Starts and ends with a
// barrier.  A round of at most kRankFlush appended candidates (the common
// case once the k best are established, and in small scans) is merged by
// counting every element's new position directly -- its rank among the
// sorted k (a binary search, or its own slot) plus the appended candidates
// better than it -- and writing it there: three barriers, where a bitonic
// sort of the same elements takes one per stage (15 for 32 elements), and the
// barriers of a 1024-thread block are the expensive part.  Larger rounds use
// the merge tree above when k <= kTreeK, else the bitonic sort, whose cost
// does not grow with the round as fast as the direct count does.
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
        } else if (k <= kTreeK && topk_flush_tree(t, k, added)) {
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

// ---- merging published lists (in the last CTA to publish)
//
// Every published list is sorted best first (it comes from a flushed or
// merged TopK).  After a merge the slots past k are unspecified; every user
// re-initialises (topk_init) before offering again.

// Slots [0, m) := the m published candidates; each thread issues all of its
// loads (two 16-byte loads per candidate) before its stores.
__device__ __forceinline__ void topk_load_cands(TopK& t, const Cand* cand, int m)
{
    const int stride = (int)blockDim.x;
    for (int i0 = threadIdx.x; i0 < m; i0 += 2 * stride) {
        const int i1 = i0 + stride;
        const ulonglong2* s0 = reinterpret_cast<const ulonglong2*>(cand + i0);
        const ulonglong2 a0 = __ldcg(s0), b0 = __ldcg(s0 + 1);
        ulonglong2 a1 = make_ulonglong2(0, 0), b1 = make_ulonglong2(0, 0);
        if (i1 < m) {
            const ulonglong2* s1 = reinterpret_cast<const ulonglong2*>(cand + i1);
            a1 = __ldcg(s1);
            b1 = __ldcg(s1 + 1);
        }
        t.key[i0] = a0.x;
        t.idx[i0] = (int64_t)a0.y;
        t.pay0[i0] = b0.x;
        t.pay1[i0] = b0.y;
        if (i1 < m) {
            t.key[i1] = a1.x;
            t.idx[i1] = (int64_t)a1.y;
            t.pay0[i1] = b1.x;
            t.pay1[i1] = b1.y;
        }
    }
}

// Lists of at most kTournamentK candidates are merged by warp tournaments:
// lane l of a warp holds the current head of list l; each round the warp
// finds the best head with a max-reduction of the keys' upper words and a
// ballot (ties, rare, fall through to the lower word and then the index),
// and the winning lane writes its head out and advances.  k rounds of a few
// dependent steps, where ranking every candidate by binary searches in every
// other list reads shared memory at scattered addresses and takes several
// times longer.  Up to 32 x 32 lists: warp w merges lists [32 w, 32 w + 32)
// and warp 0 then merges the warps' results.  (One warp holding several
// lists per lane, rescanning its heads after each win, measured slower.)
constexpr int kTournamentK = 16;

// Best (key descending, index ascending) over the warp; returns its lane in
// every lane.  Every lane must call it (warp-uniform branches only).
__device__ __forceinline__ int warp_best_lane(uint64_t key, int64_t idx)
{
    const unsigned full = 0xffffffffu;
    const uint32_t kh = (uint32_t)(key >> 32);
    const uint32_t mh = __reduce_max_sync(full, kh);
    unsigned c = __ballot_sync(full, kh == mh);
    if (__popc(c) > 1) {
        const bool in = kh == mh;
        const uint32_t kl = in ? (uint32_t)key : 0u;
        const uint32_t ml = __reduce_max_sync(full, kl);
        c = __ballot_sync(full, in && kl == ml);
        if (__popc(c) > 1) {                 // equal keys: the smallest index
            const bool in2 = in && kl == ml;
            const uint64_t u = (uint64_t)idx;
            const uint32_t ih = in2 ? (uint32_t)(u >> 32) : 0xffffffffu;
            const uint32_t mih = __reduce_min_sync(full, ih);
            c = __ballot_sync(full, in2 && ih == mih);
            if (__popc(c) > 1) {
                const bool in3 = in2 && ih == mih;
                const uint32_t il = in3 ? (uint32_t)u : 0xffffffffu;
                const uint32_t mil = __reduce_min_sync(full, il);
                c = __ballot_sync(full, in3 && il == mil);
            }
        }
    }
    return __ffs(c) - 1;
}

// One warp merges `lists` (<= 32) sorted lists of k slots at base + l * k
// into slots [out0, out0 + k), which must hold sentinels beforehand.
__device__ __forceinline__ void topk_tournament(TopK& t, int k, int lists, int base, int out0)
{
    const int lane = threadIdx.x & 31;
    int pos = 0;
    uint64_t hk = kSentinelKey;
    int64_t hi = kSentinelIndex;
    if (lane < lists) {
        hk = t.key[base + lane * k];
        hi = t.idx[base + lane * k];
    }
    for (int r = 0; r < k; ++r) {
        if (__ballot_sync(0xffffffffu, hi != kSentinelIndex) == 0u) break;   // all exhausted
        if (lane == warp_best_lane(hk, hi)) {
            const int j = base + lane * k + pos;
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

// Threads i < m rank candidate base + i by counting the candidates of
// [base, base + m) better than it and write it to out0 + rank if the rank is
// below k (ranks are distinct: the order is strict; sentinels are not
// placed, so [out0, out0 + k) must hold sentinels beforehand).  Every thread
// reads the same candidate at the same time (shared-memory broadcasts).
constexpr int kRankMerge = 256;

__device__ __forceinline__ void topk_rank_small(TopK& t, int k, int base, int m, int out0)
{
    const int i = threadIdx.x;
    if (i >= m) return;
    const uint64_t ck = t.key[base + i];
    const int64_t ci = t.idx[base + i];
    if (ci == kSentinelIndex) return;
    int r = 0;
    for (int j = 0; j < m; ++j) r += better(t.key[base + j], t.idx[base + j], ck, ci) ? 1 : 0;
    if (r < k) {
        t.key[out0 + r] = ck;
        t.idx[out0 + r] = ci;
        t.pay0[out0 + r] = t.pay0[base + i];
        t.pay1[out0 + r] = t.pay1[base + i];
    }
}

// Whether `lists` sorted lists of k slots fit the tournament merge.
__device__ __forceinline__ bool topk_tournament_fits(int k, int64_t lists)
{
    const int64_t w1 = (lists + 31) >> 5;
    return k <= kTournamentK && w1 <= 32 && w1 <= (int64_t)(blockDim.x >> 5) &&
           lists * k + (w1 > 1 ? w1 * k : 0) + k <= kTopkCap;
}

// Merge of m / k published lists into slots [0, k), when they fit the
// shared slots (else returns false, having done nothing): by the tournament
// for k <= kTournamentK, by the merge tree for k <= kTreeK, else by ranks --
// every candidate's final position is its position in its own list plus the
// number of candidates of each other list that are better (a binary search
// per list), the first k positions written to the upper half of the slots,
// then moved down (the order is strict, so positions never collide;
// sentinels are not placed).
static __device__ __noinline__ bool topk_merge_sorted(TopK t, int k, const Cand* cand, int64_t m)
{
    constexpr int kHalf = kTopkCap / 2;
    if (m % k != 0 || m > kTopkCap || k > kHalf) return false;
    const int lists = (int)(m / k);
    if (topk_tournament_fits(k, lists)) {
        const int w1 = (lists + 31) >> 5;                   // first-round warps
        const int out1 = (int)m;                            // their lists
        const int out2 = out1 + (w1 > 1 ? w1 * k : 0);      // the final list
        topk_load_cands(t, cand, (int)m);
        for (int i = out1 + threadIdx.x; i < out2 + k; i += blockDim.x) topk_clear_slot(t, i);
        __syncthreads();
        const int warp = (int)(threadIdx.x >> 5);
        if (w1 > 1) {
            if (warp < w1)
                topk_tournament(t, k, min(32, lists - 32 * warp), 32 * warp * k, out1 + warp * k);
            __syncthreads();
        }
        // the last level: few candidates are ranked directly, in parallel
        // (every thread counts the candidates better than its own: k rounds
        // of a tournament cost more below kRankMerge candidates)
        const int last_base = w1 > 1 ? out1 : 0;
        const int last_m = w1 > 1 ? w1 * k : (int)m;
        if (last_m <= kRankMerge && last_m <= (int)blockDim.x)
            topk_rank_small(t, k, last_base, last_m, out2);
        else if (warp == 0)
            topk_tournament(t, k, w1 > 1 ? w1 : lists, last_base, out2);
        __syncthreads();
        if ((int)threadIdx.x < k) {                         // [out2, out2 + k) -> [0, k), disjoint
            const int i = threadIdx.x;
            t.key[i] = t.key[out2 + i];
            t.idx[i] = t.idx[out2 + i];
            t.pay0[i] = t.pay0[out2 + i];
            t.pay1[i] = t.pay1[out2 + i];
        }
        if (threadIdx.x == 0) t.misc[0] = 0;
        __syncthreads();
        return true;
    }
    if (k <= kTreeK && m <= kHalf) {
        topk_load_cands(t, cand, (int)m);
        __syncthreads();
        const TreeSpan sp = tree_span(0, kHalf, k, lists, k);
        merge_tree(t, 0, kHalf, k, lists, k);
        if (sp.res != 0) {                                  // [kHalf, kHalf + k) -> [0, k)
            uint64_t ck = 0, cp0 = 0, cp1 = 0;
            int64_t ci = 0;
            const bool mover = (int)threadIdx.x < k;
            if (mover) {
                ck = t.key[kHalf + threadIdx.x];
                ci = t.idx[kHalf + threadIdx.x];
                cp0 = t.pay0[kHalf + threadIdx.x];
                cp1 = t.pay1[kHalf + threadIdx.x];
            }
            __syncthreads();
            if (mover) {
                t.key[threadIdx.x] = ck;
                t.idx[threadIdx.x] = ci;
                t.pay0[threadIdx.x] = cp0;
                t.pay1[threadIdx.x] = cp1;
            }
        }
        if (threadIdx.x == 0) t.misc[0] = 0;
        __syncthreads();
        return true;
    }
    if (m > kHalf) return false;
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
// holds the final list in slots [0, k).  When the whole grid's lists fit one
// tournament merge, the groups are skipped: every CTA publishes on
// tickets[0] and the last one merges all lists (one publication and one
// merge fewer on the critical path).
__device__ __forceinline__ bool topk_publish_two_level(TopK& t, int k, Cand* cand,
                                                       Cand* group_lists, unsigned int* tickets)
{
    if (topk_tournament_fits(k, gridDim.x)) {
        if (!topk_publish_slot(t, k, cand, blockIdx.x, gridDim.x, tickets)) return false;
        topk_merge_published(t, k, cand, (int64_t)gridDim.x * k);
        return true;
    }
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
