// rerank.cu -- exact Dice re-ranking of the prefilter's candidates.
//
// The candidates of each query are scored by the same exact loop as the
// full scan (Section 2.3 of Ezhov et al. 2022: Dice at both thresholds,
// added, largest wins), so the returned hits carry exact counts and binary64
// scores; only which entries are looked at comes from the prefilter.
//
// Work items are (query, slice of its candidates).  Each item gathers its
// candidates' planes with the shared count loop of scan_core.cuh (patient
// words in registers), keeps a running top-k, publishes it to the query's
// scratch row, and the last item of a query (per-query atomic ticket, no
// spinning) merges the slices into the query's k hits.
//
// Dense items all cost the same and the grid walks them round-robin.  Sparse
// items cost in proportion to their query's support, which varies thirty-fold
// between patients; there the CTAs take items from a global counter, largest
// support first (each CTA ranks the queries by support length in shared
// memory, the same order in every CTA), so the small items fill the tail.
#include "kernels.h"
#include "scan_core.cuh"
#include "topk.cuh"

namespace dbq {
namespace {

constexpr int kGroupMax = 1024;
constexpr int kOrderMax = 512;     // queries ranked by support for the sparse order

// Largest support first, ties by query index: rank of query q among all.
__device__ __forceinline__ void rank_by_support(const uint32_t* sup_lens, int nq, int* cost,
                                                int* order)
{
    for (int q = threadIdx.x; q < nq; q += blockDim.x)
        cost[q] = (int)(sup_lens[2 * q] + sup_lens[2 * q + 1]);
    __syncthreads();
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const int c = cost[q];
        int r = 0;
        for (int j = 0; j < nq; ++j) {
            const int cj = cost[j];
            r += (cj > c || (cj == c && j < q)) ? 1 : 0;
        }
        order[r] = q;
    }
    __syncthreads();
}

template <int U, int EPI, bool kSparse>
__global__ void __launch_bounds__(kScanThreads, 1)
rerank_kernel(const RerankArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TopK tk;
    unsigned char* after_topk = topk_carve(tk, smem_raw);
    uint32_t* icnt = reinterpret_cast<uint32_t*>(after_topk);                  // [kGroupMax][2]
    int* next = reinterpret_cast<int*>(after_topk + (size_t)kGroupMax * 2 * sizeof(uint32_t));
    int* order = next + 4;                                                     // [kOrderMax]
    int* cost = order + kOrderMax;                                              // [kOrderMax]
    unsigned char* cache_raw = reinterpret_cast<unsigned char*>(cost + kOrderMax);
    __shared__ int s_item;
    const int tid = threadIdx.x;
    const int per = (a.c + a.slices - 1) / a.slices;
    const int items = a.nq * a.slices;
    const uint2* ecount2 = reinterpret_cast<const uint2*>(a.ecount);
    // every CTA makes exactly one failing grab, so items + grid grabs return
    // the counter to zero for the next launch
    const bool dynamic = kSparse && a.sched != nullptr;
    if (dynamic) rank_by_support(a.sup_lens, a.nq, cost, order);
    for (int iter = 0;; ++iter) {
        if (dynamic) {
            if (tid == 0) s_item = (int)atomicInc(a.sched, (unsigned)(items + gridDim.x - 1));
            __syncthreads();
        }
        const int item = dynamic ? s_item : (int)blockIdx.x + iter * (int)gridDim.x;
        if (item >= items) break;
        const int q = dynamic ? order[item / a.slices] : item / a.slices;
        const int sl = item % a.slices;
        const int first = sl * per;
        const int gn = (a.c - first) < per ? (a.c - first) : per;
        const int32_t* list = a.cand + (int64_t)q * a.c + first;
        const uint4* patient = a.patients + (int64_t)q * 2 * a.wp4;
        const uint32_t P1 = a.pcounts[2 * q];
        const uint32_t P2 = a.pcounts[2 * q + 1];
        topk_init(tk);
        for (int i = tid; i < 2 * kGroupMax; i += kScanThreads) icnt[i] = 0u;
        if (tid == 0) *next = 0;
        __syncthreads();
        if (gn > 0) {
            Support sup;
            bool warp_mode = false;
            SupportCache cache;
            if (kSparse) {
                sup.list1 = a.sup_lists + (int64_t)q * 2 * a.wp4;
                sup.list2 = sup.list1 + a.wp4;
                sup.len = a.sup_lens + 2 * q;
                warp_mode = load_support_cache(cache_raw, patient, a.wp4, sup, cache);
            }
            if (warp_mode)
                count_group_warps(a.planes, a.wp4, list, 0, gn, icnt, cache, next);
            else
                count_group<U, EPI, kSparse>(a.planes, a.wp4, a.chunk4, a.nchunks, patient, list,
                                             0, gn, icnt, sup);
        }
        __syncthreads();
        for (int i = tid; i < gn; i += kScanThreads) {
            const int64_t e = list[i];
            const uint32_t I1 = icnt[2 * i], I2 = icnt[2 * i + 1];
            const uint2 E = ecount2[e];
            topk_offer_counts(tk, a.k, I1, I2, E.x, E.y, P1, P2, e);
        }
        topk_flush(tk, a.k);
        Cand* rows = a.scratch + (int64_t)q * a.slices * a.k;
        if (topk_publish_slot(tk, a.k, rows, sl, a.slices, a.tickets + q)) {
            topk_merge_published(tk, a.k, rows, (int64_t)a.slices * a.k);
            for (int j = tid; j < a.k; j += kScanThreads) {
                Hit h;
                h.index = tk.idx[j];
                h.score = key_score(tk.key[j]);
                h.i1 = (uint32_t)(tk.pay0[j] & 0xffffffffu);
                h.i2 = (uint32_t)(tk.pay0[j] >> 32);
                h.e1 = (uint32_t)(tk.pay1[j] & 0xffffffffu);
                h.e2 = (uint32_t)(tk.pay1[j] >> 32);
                h.p1 = P1;
                h.p2 = P2;
                a.hits[(int64_t)q * a.k + j] = h;
            }
        }
        __syncthreads();   // the shared top-k is reused by the next item
    }
}

}  // namespace

cudaError_t launch_rerank(const RerankArgs& a, cudaStream_t stream)
{
    if (a.nq < 1 || a.c < 1 || a.k < 1 || a.k > a.c || a.slices < 1 ||
        (a.c + a.slices - 1) / a.slices > kGroupMax)
        return cudaErrorInvalidValue;
    if (a.sched && (!a.sup_lists || a.nq > kOrderMax)) return cudaErrorInvalidValue;
    const size_t smem = topk_smem_bytes() + (size_t)kGroupMax * 2 * sizeof(uint32_t) + 16 +
                        (size_t)2 * kOrderMax * sizeof(int) +
                        (a.sup_lists ? kSupportCacheBytes : 0);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int items = a.nq * a.slices;
    const int grid = items < sms ? items : sms;
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
        kern<<<grid, kScanThreads, smem, stream>>>(a);
        return cudaGetLastError();
    };
    if (a.sup_lists) {
        if (a.chunk4 <= kScanThreads) return run(rerank_kernel<1, 4, true>);
        return run(rerank_kernel<2, 2, true>);
    }
    if (a.chunk4 <= kScanThreads) return run(rerank_kernel<1, 4, false>);
    return run(rerank_kernel<2, 2, false>);
}

}  // namespace dbq
