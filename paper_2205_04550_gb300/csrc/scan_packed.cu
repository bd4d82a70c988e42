// scan_packed.cu -- the brute-force query over a bit-packed database, fused
// with scoring and top-k selection in one persistent launch.
//
// Ezhov et al. (2022), Section 2.3: the baseline search loops over every
// database entry and compares it with the patient by Dice at the two
// thresholds; the two Dice values are added and the best-scoring entry wins.
// With masks stored as bit planes, |P_k n E_k| is a sum of popcounts of the
// AND of the patient's and the entry's words; |E_k| was counted at build
// time and |P_k| when the patient was packed.
//
// GB300 mapping (one CTA of 1024 threads per SM, persistent):
//   * CTA b owns the contiguous entry range [b*N/G, (b+1)*N/G).
//   * The patient's planes are split into chunks of 2 x 32 KiB.  Within a
//     chunk, thread t always handles the same two 16-byte positions of each
//     plane, so it holds the patient's words for them in registers; it then
//     streams those positions of each of its entries from HBM with 128-bit
//     no-L1-allocate loads (every database byte is read exactly once per
//     query, two entries in flight), ANDs, POPCs, reduces across the warp
//     with redux.sync and adds the warp's sum into a per-entry shared
//     counter.
//   * When every chunk of a group of entries is done the CTA knows their
//     exact I_1, I_2, computes the binary64 scores and keeps a running
//     top-k in shared memory (topk.cuh; order: score desc, index asc).
//   * Each CTA writes its list to scratch; the last CTA to finish (atomic
//     ticket, no spinning; in groups of CTAs first for larger k) merges the
//     lists and writes the k hits.
//   * With counts_in (the word-major sparse scan) the counts come from
//     memory instead of the planes; scoring and selection are the same.
#include "kernels.h"
#include "scan_core.cuh"
#include "topk.cuh"

namespace dbq {
namespace {

constexpr int kThreads = kScanThreads;
constexpr int kGroup = 1024;        // entries whose counters live in shared memory
static_assert(kGroup == kThreads, "one entry of a group per thread when scoring");
constexpr int kMaxChunk4 = 2048;    // uint4 per plane per chunk = 2 per thread

template <int U, int EPI, bool kSparse>
__global__ void __launch_bounds__(kThreads, 1)
scan_packed_kernel(const ScanPackedArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TopK tk;
    unsigned char* after_topk = topk_carve(tk, smem_raw);
    uint32_t* icnt = reinterpret_cast<uint32_t*>(after_topk);                  // [kGroup][2]
    unsigned char* cache_raw = after_topk + (size_t)kGroup * 2 * sizeof(uint32_t) + 16;
    int* next = reinterpret_cast<int*>(after_topk + (size_t)kGroup * 2 * sizeof(uint32_t));
    const int tid = threadIdx.x;
    const int k = a.k;
    const bool want_topk = a.hits != nullptr;
    const int64_t e_begin = (int64_t)blockIdx.x * a.n / gridDim.x;
    const int64_t e_end = ((int64_t)blockIdx.x + 1) * a.n / gridDim.x;
    const uint32_t P1 = a.pcount[0];
    const uint32_t P2 = a.pcount[1];
    const uint2* ecount2 = reinterpret_cast<const uint2*>(a.ecount);
    Support sup;
    sup.list1 = a.sup_list;
    sup.list2 = a.sup_list + a.wp4;
    sup.len = a.sup_len;
    SupportCache cache;
    bool warp_mode = false;
    if (kSparse) warp_mode = load_support_cache(cache_raw, a.patient, a.wp4, sup, cache);

    topk_init(tk);

    for (int64_t g0 = e_begin; g0 < e_end; g0 += kGroup) {
        const int gn = (int)((e_end - g0) < kGroup ? (e_end - g0) : kGroup);
        for (int i = tid; i < 2 * kGroup; i += kThreads) icnt[i] = 0u;
        if (tid == 0) *next = 0;
        // The entries' mask sizes are fetched before the count, so the
        // scoring after it does not wait on memory for them (kGroup ==
        // kThreads: one entry per thread): into registers in the dense scan,
        // into L2 in the sparse one, whose counts have no register to spare.
        const bool mine = want_topk && tid < gn;
        uint2 E = make_uint2(0u, 0u);
        if (!kSparse && mine) E = ecount2[g0 + tid];
        if (kSparse && mine) asm volatile("prefetch.global.L2 [%0];" ::"l"(ecount2 + g0 + tid));
        __syncthreads();
        if (a.counts_in) {
            for (int i = tid; i < 2 * gn; i += kThreads) icnt[i] = a.counts_in[2 * g0 + i];
        } else if (warp_mode) {
            count_group_warps(a.planes, a.wp4, nullptr, g0, gn, icnt, cache, next);
        } else {
            count_group<U, EPI, kSparse>(a.planes, a.wp4, a.chunk4, a.nchunks, a.patient,
                                         nullptr, g0, gn, icnt, sup);
        }
        __syncthreads();   // the group's counters are complete
        for (int i = tid; i < gn; i += kThreads) {
            const int64_t e = g0 + i;
            const uint32_t I1 = icnt[2 * i];
            const uint32_t I2 = icnt[2 * i + 1];
            const uint2 Ec = kSparse || !want_topk ? ecount2[e] : E;
            if (a.counts_out)
                reinterpret_cast<uint4*>(a.counts_out)[e] = make_uint4(I1, I2, Ec.x, Ec.y);
            if (want_topk)
                topk_offer_counts(tk, k, I1, I2, Ec.x, Ec.y, P1, P2, e);
        }
        if (want_topk) topk_flush(tk, k);
        else __syncthreads();
    }
    if (!want_topk) return;
    if (a.group_lists) {
        if (!topk_publish_two_level(tk, k, a.cand, a.group_lists, a.tickets)) return;
    } else {
        if (!topk_publish(tk, k, a.cand, a.ticket)) return;
        topk_merge_published(tk, k, a.cand, (int64_t)gridDim.x * k);
    }
    for (int j = tid; j < k; j += kThreads) {
        Hit h;
        h.index = tk.idx[j];
        h.score = key_score(tk.key[j]);
        h.i1 = (uint32_t)(tk.pay0[j] & 0xffffffffu);
        h.i2 = (uint32_t)(tk.pay0[j] >> 32);
        h.e1 = (uint32_t)(tk.pay1[j] & 0xffffffffu);
        h.e2 = (uint32_t)(tk.pay1[j] >> 32);
        h.p1 = P1;
        h.p2 = P2;
        a.hits[j] = h;
    }
}

}  // namespace

size_t scan_packed_smem(int chunk4)
{
    (void)chunk4;   // the patient lives in registers
    return topk_smem_bytes() + (size_t)kGroup * 2 * sizeof(uint32_t) + 16;
}

void scan_packed_chunking(int wp4, int* chunk4, int* nchunks)
{
    int nc = (wp4 + kMaxChunk4 - 1) / kMaxChunk4;
    if (nc < 1) nc = 1;
    int c4 = (wp4 + nc - 1) / nc;
    if (c4 < 1) c4 = 1;
    *chunk4 = c4;
    *nchunks = (wp4 + c4 - 1) / c4;
}

int scan_packed_grid(int device)
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        sms <= 0)
        sms = 1;
    return sms;   // one 1024-thread CTA per SM
}

cudaError_t launch_scan_packed(const ScanPackedArgs& a, int grid, cudaStream_t stream)
{
    // the sparse variant also holds the patient's support in shared memory
    const size_t smem = scan_packed_smem(a.chunk4) + (a.sup_list ? kSupportCacheBytes : 0);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
        kern<<<grid, kThreads, smem, stream>>>(a);
        return cudaGetLastError();
    };
    if (a.sup_list) {
        if (a.chunk4 <= kThreads) return run(scan_packed_kernel<1, 4, true>);
        return run(scan_packed_kernel<2, 2, true>);
    }
    if (a.chunk4 <= kThreads) return run(scan_packed_kernel<1, 4, false>);
    return run(scan_packed_kernel<2, 2, false>);
}

}  // namespace dbq
