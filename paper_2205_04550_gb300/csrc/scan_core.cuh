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

// icnt[2 * i + k] += I_k of entry i of the group (i < gn); the group's
// entries are list[g0 + i] when `list` is given, else g0 + i.  icnt must be
// zeroed and visible (barrier) before the call; the call ends without a
// barrier.
template <int U, int EPI>
__device__ __forceinline__ void count_group(const uint4* __restrict__ planes, int wp4, int chunk4,
                                            int nchunks, const uint4* __restrict__ patient,
                                            const int32_t* __restrict__ list, int64_t g0, int gn,
                                            uint32_t* icnt)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    for (int c = 0; c < nchunks; ++c) {
        const int c0 = c * chunk4;
        const int clen = (wp4 - c0) < chunk4 ? (wp4 - c0) : chunk4;
        uint4 pa[U], pb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = tid + u * kScanThreads;
            pa[u] = (j < clen) ? patient[c0 + j] : make_uint4(0, 0, 0, 0);
            pb[u] = (j < clen) ? patient[wp4 + c0 + j] : make_uint4(0, 0, 0, 0);
        }
        for (int i0 = 0; i0 < gn; i0 += EPI) {
            uint4 x[EPI][U], y[EPI][U];
#pragma unroll
            for (int q = 0; q < EPI; ++q) {
                const bool ev = (i0 + q) < gn;
                int64_t e = g0 + i0 + q;
                if (list && ev) e = list[e];
                const uint4* p0 = planes + e * 2 * wp4 + c0;
                const uint4* p1 = p0 + wp4;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = tid + u * kScanThreads;
                    if (ev && j < clen) {
                        x[q][u] = ld_stream(p0 + j);
                        y[q][u] = ld_stream(p1 + j);
                    } else {
                        x[q][u] = make_uint4(0, 0, 0, 0);
                        y[q][u] = make_uint4(0, 0, 0, 0);
                    }
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

}  // namespace dbq
