// scan_core.cuh -- the exact intersection counts of a group of entries
// against one patient, shared by the fused packed scan and the re-ranking of
// prefilter candidates.
//
// |P_k n E_k| = sum over words of popc(patient_k[w] & entry_k[w]) (the
// Dice numerator of Section 2.3, Ezhov et al. 2022).  The planes are split
// into chunks of at most 2 x 1024 16-byte words; within a chunk thread t
// handles the positions t + u * 1024 (u < U) of both planes, keeps the
// patient's words for them in registers, and streams those positions of EPI
// entries at a time with 128-bit no-L1-allocate loads.  Warp sums are
// reduced with redux.sync and added into per-entry shared counters.
#pragma once

#include "common.cuh"

namespace dbq {

constexpr int kScanThreads = 1024;

// Patient support lists: for plane k, the 16-byte word offsets of the
// patient's non-zero 64-byte granules (four consecutive offsets per
// granule, ascending), and their count.  Words outside the list are zero in
// the patient, so they add nothing to |P_k n E_k| and need not be read.
struct Support {
    const uint32_t* list1;   // [wp4] offsets into plane 1
    const uint32_t* list2;   // [wp4] offsets into plane 2
    const uint32_t* len;     // [2]  list lengths
};

// icnt[2 * i + k] += I_k of entry i of the group (i < gn); the group's
// entries are list[g0 + i] when `list` is given, else g0 + i.  With kSparse
// the positions visited are the patient's support lists instead of all
// words.  icnt must be zeroed and visible (barrier) before the call; the call
// ends without a barrier.
template <int U, int EPI, bool kSparse = false>
__device__ __forceinline__ void count_group(const uint4* __restrict__ planes, int wp4, int chunk4,
                                            int nchunks, const uint4* __restrict__ patient,
                                            const int32_t* __restrict__ list, int64_t g0, int gn,
                                            uint32_t* icnt, Support sup = Support{})
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    int len1 = wp4, len2 = wp4;
    if (kSparse) {
        len1 = (int)sup.len[0];
        len2 = (int)sup.len[1];
        const int longest = len1 > len2 ? len1 : len2;
        nchunks = (longest + chunk4 - 1) / chunk4;
    }
    for (int c = 0; c < nchunks; ++c) {
        const int c0 = c * chunk4;
        const int clen1 = (len1 - c0) < chunk4 ? (len1 - c0) : chunk4;
        const int clen2 = (len2 - c0) < chunk4 ? (len2 - c0) : chunk4;
        uint4 pa[U], pb[U];
        uint32_t o1[U], o2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = tid + u * kScanThreads;
            o1[u] = (j < clen1) ? (kSparse ? sup.list1[c0 + j] : (uint32_t)(c0 + j)) : 0u;
            o2[u] = (j < clen2) ? (kSparse ? sup.list2[c0 + j] : (uint32_t)(c0 + j)) : 0u;
            pa[u] = (j < clen1) ? patient[o1[u]] : make_uint4(0, 0, 0, 0);
            pb[u] = (j < clen2) ? patient[wp4 + o2[u]] : make_uint4(0, 0, 0, 0);
        }
        for (int i0 = 0; i0 < gn; i0 += EPI) {
            uint4 x[EPI][U], y[EPI][U];
#pragma unroll
            for (int q = 0; q < EPI; ++q) {
                const bool ev = (i0 + q) < gn;
                int64_t e = g0 + i0 + q;
                if (list && ev) e = list[e];
                const uint4* p0 = planes + e * 2 * wp4;
                const uint4* p1 = p0 + wp4;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = tid + u * kScanThreads;
                    x[q][u] = (ev && j < clen1) ? ld_stream(p0 + o1[u]) : make_uint4(0, 0, 0, 0);
                    y[q][u] = (ev && j < clen2) ? ld_stream(p1 + o2[u]) : make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int q = 0; q < EPI; ++q) {
                uint32_t a1 = 0, a2 = 0;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    a1 += popc_and4(x[q][u], pa[u]);
                    a2 += popc_and4(y[q][u], pb[u]);
                }
                a1 = __reduce_add_sync(0xffffffffu, a1);
                a2 = __reduce_add_sync(0xffffffffu, a2);
                if (lane == 0 && (i0 + q) < gn) {
                    if (a1) atomicAdd(&icnt[2 * (i0 + q)], a1);
                    if (a2) atomicAdd(&icnt[2 * (i0 + q) + 1], a2);
                }
            }
        }
    }
}

// ---- sparse scan, one warp per entry
//
// When the patient's support is small, a CTA-wide pass per entry leaves most
// threads idle.  Instead the support (word offsets and the patient's words
// there) is cached in shared memory once, and each warp scans whole entries:
// lane l visits support positions l, l + 32, ... of both planes, four loads
// in flight per plane, and the warp's sums go straight to the entry's
// counters (no atomics: one warp owns an entry).

// Shared-memory cache of one patient's support: 20 bytes per position.
// Positions [0, len1) belong to plane 1, [len1, len1 + len2) to plane 2;
// off[] holds word offsets from the start of an entry (plane 2 offsets
// include the plane stride), pw[] the patient's words there.
struct SupportCache {
    const uint32_t* off;
    const uint4* pw;
    int len1;
    int len2;
};

constexpr int kSupportCacheBytes = 150 * 1024;
constexpr int kSupportCachePositions = kSupportCacheBytes / 20;

// Fill the cache from the support lists (all threads; ends with a barrier).
// Returns false, without filling, if the support does not fit.
__device__ __forceinline__ bool load_support_cache(unsigned char* raw, const uint4* patient,
                                                   int wp4, const Support& sup, SupportCache& c)
{
    const int l1 = (int)sup.len[0], l2 = (int)sup.len[1];
    if (l1 + l2 > kSupportCachePositions) return false;
    uint4* pw = reinterpret_cast<uint4*>(raw);                 // [l1 + l2]
    uint32_t* off = reinterpret_cast<uint32_t*>(pw + (l1 + l2));
    for (int j = threadIdx.x; j < l1 + l2; j += blockDim.x) {
        const uint32_t o = j < l1 ? sup.list1[j] : (uint32_t)wp4 + sup.list2[j - l1];
        off[j] = o;
        pw[j] = patient[o];
    }
    c.off = off;
    c.pw = pw;
    c.len1 = l1;
    c.len2 = l2;
    __syncthreads();
    return true;
}

// icnt[2 * i + k] = I_k of entry i of the group (written, not added); the
// entries are list[g0 + i] or g0 + i.  Warps take entries from the shared
// counter `next` (zeroed by the caller before a barrier); lane l visits
// positions l, l + 32, ... of both planes, eight loads in flight.  Ends
// without a barrier.
__device__ __forceinline__ void count_group_warps(const uint4* __restrict__ planes, int wp4,
                                                  const int32_t* __restrict__ list, int64_t g0,
                                                  int gn, uint32_t* icnt, const SupportCache& c,
                                                  int* next)
{
    const int lane = threadIdx.x & 31;
    const int total = c.len1 + c.len2;
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(next, 1);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= gn) break;
        int64_t e = g0 + i;
        if (list) e = list[e];
        const uint4* base = planes + e * 2 * wp4;
        uint32_t a1 = 0, a2 = 0;
        // eight predicated loads per iteration, so the last partial round
        // also has all of its loads in flight at once
        for (int j = lane; j < total; j += 8 * 32) {
            uint4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int p = j + 32 * u;
                v[u] = p < total ? ld_stream(base + c.off[p]) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int p = j + 32 * u;
                if (p < total) {
                    const uint32_t cnt = popc_and4(v[u], c.pw[p]);
                    if (p < c.len1) a1 += cnt;
                    else a2 += cnt;
                }
            }
        }
        const uint32_t s1 = __reduce_add_sync(0xffffffffu, a1);
        const uint32_t s2 = __reduce_add_sync(0xffffffffu, a2);
        if (lane == 0) {
            icnt[2 * i] = s1;
            icnt[2 * i + 1] = s2;
        }
    }
}

}  // namespace dbq
