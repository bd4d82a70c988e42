// scan_tasks.cu -- many exact queries, against several bit-packed databases
// of different resolutions, in one persistent launch.
//
// Each query is the brute-force loop of Section 2.3 (Ezhov et al. 2022) over
// its database.  A query is split into slices of its entries; the work items
// (query, slice) of all queries form one list that the CTAs of a persistent
// grid take from a global counter, so queries of different sizes balance
// over the GPU.  An item counts its entries with the shared count loop
// (dense, or restricted to the patient's support lists), keeps a running
// top-k, publishes it to the query's scratch row; the last item of a query
// (per-query atomic ticket, no spinning) merges the slices into its k hits.
//
// The host splits queries into slices in proportion to their databases'
// dense bytes.  A sparse query reads only its patient's support, which the
// host does not know when it enqueues the launch (the support lists are
// built on the device just before), and supports differ thirty-fold; for
// launches with sparse queries a one-CTA kernel therefore re-orders the
// items on the device, longest first, before the scan starts.
#include "kernels.h"
#include "scan_core.cuh"
#include "topk.cuh"

namespace dbq {
namespace {

constexpr int kGroup = 1024;

template <int U, int EPI, bool kSparse>
__device__ __forceinline__ void count_task(const QueryTask& t, int64_t g0, int gn, uint32_t* icnt)
{
    if (kSparse && t.sup_list) {
        Support sup;
        sup.list1 = t.sup_list;
        sup.list2 = t.sup_list + t.wp4;
        sup.len = t.sup_len;
        count_group<U, EPI, true>(t.planes, t.wp4, t.chunk4, t.nchunks, t.patient, nullptr, g0,
                                  gn, icnt, sup);
    } else {
        count_group<U, EPI, false>(t.planes, t.wp4, t.chunk4, t.nchunks, t.patient, nullptr, g0,
                                   gn, icnt);
    }
}

// kSparse: the launch holds queries with support lists (warp-per-entry path
// compiled in); the dense-only instantiation keeps its registers for the
// CTA-wide loop.
template <bool kSparse>
__global__ void __launch_bounds__(kScanThreads, 1)
scan_tasks_kernel(const QueryTask* __restrict__ tasks, const int2* __restrict__ items, int nitems,
                  unsigned int* __restrict__ next_item)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TopK tk;
    unsigned char* after_topk = topk_carve(tk, smem_raw);
    uint32_t* icnt = reinterpret_cast<uint32_t*>(after_topk);                  // [kGroup][2]
    int* next = reinterpret_cast<int*>(after_topk + (size_t)kGroup * 2 * sizeof(uint32_t));
    unsigned char* cache_raw = after_topk + (size_t)kGroup * 2 * sizeof(uint32_t) + 16;
    __shared__ int item_s;
    __shared__ QueryTask task_s;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) item_s = (int)atomicAdd(next_item, 1u);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= nitems) break;
        const int2 it = items[item];
        if (tid == 0) task_s = tasks[it.x];
        __syncthreads();
        const QueryTask& t = task_s;
        const int sl = it.y;
        const int64_t e_begin = (int64_t)sl * t.n / t.slices;
        const int64_t e_end = ((int64_t)sl + 1) * t.n / t.slices;
        const uint32_t P1 = t.pcount[0], P2 = t.pcount[1];
        const uint2* ecount2 = reinterpret_cast<const uint2*>(t.ecount);
        topk_init(tk);
        SupportCache cache;
        bool warp_mode = false;
        if (kSparse && t.sup_list) {
            Support sup;
            sup.list1 = t.sup_list;
            sup.list2 = t.sup_list + t.wp4;
            sup.len = t.sup_len;
            warp_mode = load_support_cache(cache_raw, t.patient, t.wp4, sup, cache);
        }
        for (int64_t g0 = e_begin; g0 < e_end; g0 += kGroup) {
            const int gn = (int)((e_end - g0) < kGroup ? (e_end - g0) : kGroup);
            for (int i = tid; i < 2 * kGroup; i += kScanThreads) icnt[i] = 0u;
            if (tid == 0) *next = 0;
            __syncthreads();
            if (kSparse && warp_mode)
                count_group_warps(t.planes, t.wp4, nullptr, g0, gn, icnt, cache, next);
            else if (t.chunk4 <= kScanThreads) count_task<1, 4, kSparse>(t, g0, gn, icnt);
            else count_task<2, 2, kSparse>(t, g0, gn, icnt);
            __syncthreads();
            for (int i = tid; i < gn; i += kScanThreads) {
                const int64_t e = g0 + i;
                const uint32_t I1 = icnt[2 * i], I2 = icnt[2 * i + 1];
                const uint2 E = ecount2[e];
                topk_offer_counts(tk, t.k, I1, I2, E.x, E.y, P1, P2, e);
            }
            topk_flush(tk, t.k);
        }
        if (topk_publish_slot(tk, t.k, t.scratch, sl, t.slices, t.ticket)) {
            topk_merge_published(tk, t.k, t.scratch, (int64_t)t.slices * t.k);
            for (int j = tid; j < t.k; j += kScanThreads) {
                Hit h;
                h.index = tk.idx[j];
                h.score = key_score(tk.key[j]);
                h.i1 = (uint32_t)(tk.pay0[j] & 0xffffffffu);
                h.i2 = (uint32_t)(tk.pay0[j] >> 32);
                h.e1 = (uint32_t)(tk.pay1[j] & 0xffffffffu);
                h.e2 = (uint32_t)(tk.pay1[j] >> 32);
                h.p1 = P1;
                h.p2 = P2;
                t.hits[j] = h;
            }
        }
        __syncthreads();
    }
}

// Power-of-two class of an item's cost: its entries times the 16-byte
// words it reads per entry (both planes' support, or both whole planes).
__device__ __forceinline__ int cost_class(const QueryTask& t)
{
    const uint64_t per_entry = t.sup_list ? (uint64_t)t.sup_len[0] + t.sup_len[1]
                                          : 2ull * (uint64_t)t.wp4;
    const uint64_t entries = (uint64_t)((t.n + t.slices - 1) / t.slices);
    return 63 - __clzll((long long)(per_entry * entries + 1));
}

// Rewrites the item list with the items of the costliest classes first (an
// approximate longest-processing-time order; within a class the order is
// that of the atomic cursor, which the results do not depend on: hits are
// ordered by score and index).  One CTA.
__global__ void order_items_kernel(const QueryTask* __restrict__ tasks, int ntasks,
                                   int2* __restrict__ items)
{
    __shared__ unsigned int hist[64];
    __shared__ unsigned int cursor[64];
    if (threadIdx.x < 64) hist[threadIdx.x] = 0u;
    __syncthreads();
    for (int t = threadIdx.x; t < ntasks; t += blockDim.x)
        if (tasks[t].slices > 0)
            atomicAdd(&hist[cost_class(tasks[t])], (unsigned int)tasks[t].slices);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int run = 0;
        for (int b = 63; b >= 0; --b) {
            cursor[b] = run;
            run += hist[b];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntasks; t += blockDim.x) {
        const int sl = tasks[t].slices;
        if (sl <= 0) continue;              // a task without items (tensor-core path)
        const unsigned int pos = atomicAdd(&cursor[cost_class(tasks[t])], (unsigned int)sl);
        for (int j = 0; j < sl; ++j) items[pos + j] = make_int2(t, j);
    }
}

}  // namespace

size_t scan_tasks_smem(bool sparse)
{
    return topk_smem_bytes() + (size_t)kGroup * 2 * sizeof(uint32_t) + 16 +
           (sparse ? kSupportCacheBytes : 0);
}

cudaError_t launch_scan_tasks(const QueryTask* tasks, int ntasks, int2* items, int nitems,
                              unsigned int* next_item, int grid, bool any_sparse,
                              cudaStream_t stream)
{
    if (nitems <= 0) return cudaSuccess;
    if (any_sparse) {
        order_items_kernel<<<1, 1024, 0, stream>>>(tasks, ntasks, items);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const size_t smem = scan_tasks_smem(any_sparse);
    auto kern = any_sparse ? scan_tasks_kernel<true> : scan_tasks_kernel<false>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(next_item, 0, sizeof(unsigned int), stream);
    if (err != cudaSuccess) return err;
    kern<<<grid, kScanThreads, smem, stream>>>(tasks, items, nitems, next_item);
    return cudaGetLastError();
}

}  // namespace dbq
