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
//   * The patient's planes are split into chunks of at most 2 x 64 KiB that
//     live in shared memory; for each chunk the CTA streams the matching
//     words of each of its entries from HBM with 128-bit no-L1-allocate
//     loads (every database byte is read exactly once per query), ANDs them
//     with the shared-memory copy, POPCs, reduces across the warp with
//     redux.sync and adds the warp's sum into a per-entry shared counter.
//   * When every chunk of a group of entries is done the CTA knows their
//     exact I_1, I_2, computes the binary64 scores and keeps a running
//     top-k in shared memory (bitonic sort, order: score desc, index asc).
//   * Each CTA writes its list to scratch; the last CTA to finish (atomic
//     ticket, no spinning) merges all lists and writes the k hits.
#include "kernels.h"

namespace dbq {
namespace {

constexpr int kThreads = 1024;
constexpr int kCap = 2048;          // shared candidate buffer (running top-k + new)
constexpr int kGroup = 1024;        // entries whose counters live in shared memory
constexpr int kMaxChunk4 = 4096;    // uint4 per plane per chunk (64 KiB per plane)

struct Smem {
    uint4* pat;        // [2][chunk4]
    double* key;       // [kCap]
    int64_t* idx;      // [kCap]
    uint64_t* pay;     // [kCap]
    uint32_t* icnt;    // [kGroup][2]
    int* misc;         // [0] = appended count, [1] = is-last flag
};

__device__ __forceinline__ Smem carve(unsigned char* raw, int chunk4)
{
    Smem s;
    s.pat = reinterpret_cast<uint4*>(raw);
    unsigned char* p = raw + (size_t)2 * chunk4 * sizeof(uint4);
    s.key = reinterpret_cast<double*>(p);
    p += kCap * sizeof(double);
    s.idx = reinterpret_cast<int64_t*>(p);
    p += kCap * sizeof(int64_t);
    s.pay = reinterpret_cast<uint64_t*>(p);
    p += kCap * sizeof(uint64_t);
    s.icnt = reinterpret_cast<uint32_t*>(p);
    p += kGroup * 2 * sizeof(uint32_t);
    s.misc = reinterpret_cast<int*>(p);
    return s;
}

__device__ __forceinline__ void topk_reset(Smem& s, int from)
{
    for (int i = from + threadIdx.x; i < kCap; i += blockDim.x) {
        s.key[i] = kSentinelScore;
        s.idx[i] = kSentinelIndex;
        s.pay[i] = 0;
    }
}

// Append a candidate if it beats the current k-th best.  The k-th best does
// not change between flushes, so every thread may read it.
__device__ __forceinline__ void topk_offer(Smem& s, int k, double score, int64_t index,
                                           uint64_t payload)
{
    if (better(score, index, s.key[k - 1], s.idx[k - 1])) {
        const int pos = k + atomicAdd(&s.misc[0], 1);
        s.key[pos] = score;
        s.idx[pos] = index;
        s.pay[pos] = payload;
    }
}

// Merge the appended candidates into the running top-k (slots [0, k)).
__device__ __forceinline__ void topk_flush(Smem& s, int k)
{
    __syncthreads();
    const int added = s.misc[0];
    if (added > 0) {
        const int n2 = next_pow2(k + added);
        bitonic_sort_best_first(s.key, s.idx, s.pay, n2);   // ends with __syncthreads
        for (int i = k + threadIdx.x; i < n2; i += blockDim.x) {
            s.key[i] = kSentinelScore;
            s.idx[i] = kSentinelIndex;
            s.pay[i] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) s.misc[0] = 0;
    __syncthreads();
}

template <int U, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
scan_packed_kernel(const ScanPackedArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem s = carve(smem_raw, a.chunk4);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int k = a.k;
    const int64_t e_begin = (int64_t)blockIdx.x * a.n / gridDim.x;
    const int64_t e_end = ((int64_t)blockIdx.x + 1) * a.n / gridDim.x;
    const uint32_t P1 = a.pcount[0];
    const uint32_t P2 = a.pcount[1];
    const uint2* ecount2 = reinterpret_cast<const uint2*>(a.ecount);

    topk_reset(s, 0);
    if (tid == 0) s.misc[0] = 0;
    int loaded_chunk = -1;

    for (int64_t g0 = e_begin; g0 < e_end; g0 += kGroup) {
        const int gn = (int)((e_end - g0) < kGroup ? (e_end - g0) : kGroup);
        for (int i = tid; i < 2 * kGroup; i += kThreads) s.icnt[i] = 0u;
        for (int c = 0; c < a.nchunks; ++c) {
            const int c0 = c * a.chunk4;
            const int clen = (a.wp4 - c0) < a.chunk4 ? (a.wp4 - c0) : a.chunk4;
            if (loaded_chunk != c) {
                __syncthreads();   // nobody still reads the previous chunk
                for (int j = tid; j < clen; j += kThreads) {
                    s.pat[j] = a.patient[c0 + j];
                    s.pat[a.chunk4 + j] = a.patient[a.wp4 + c0 + j];
                }
                loaded_chunk = c;
            }
            __syncthreads();
            for (int i0 = 0; i0 < gn; i0 += EPI) {
                uint4 x[EPI][U], y[EPI][U];
#pragma unroll
                for (int q = 0; q < EPI; ++q) {
                    const bool ev = (i0 + q) < gn;
                    const uint4* p0 = a.planes + (g0 + i0 + q) * 2 * a.wp4 + c0;
                    const uint4* p1 = p0 + a.wp4;
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int j = tid + u * kThreads;
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
                        const int j = tid + u * kThreads;
                        if (j < clen) {
                            a1 += popc_and4(x[q][u], s.pat[j]);
                            a2 += popc_and4(y[q][u], s.pat[a.chunk4 + j]);
                        }
                    }
                    a1 = __reduce_add_sync(0xffffffffu, a1);
                    a2 = __reduce_add_sync(0xffffffffu, a2);
                    if (lane == 0 && (i0 + q) < gn) {
                        if (a1) atomicAdd(&s.icnt[2 * (i0 + q)], a1);
                        if (a2) atomicAdd(&s.icnt[2 * (i0 + q) + 1], a2);
                    }
                }
            }
        }
        __syncthreads();   // the group's counters are complete
        for (int i = tid; i < gn; i += kThreads) {
            const int64_t e = g0 + i;
            const uint32_t I1 = s.icnt[2 * i];
            const uint32_t I2 = s.icnt[2 * i + 1];
            const uint2 E = ecount2[e];
            if (a.counts_out) {
                reinterpret_cast<uint4*>(a.counts_out)[e] = make_uint4(I1, I2, E.x, E.y);
            }
            if (a.hits) {
                const double sc = score_rn(I1, I2, E.x, E.y, P1, P2);
                topk_offer(s, k, sc, e, (uint64_t)I1 | ((uint64_t)I2 << 32));
            }
        }
        if (a.hits) topk_flush(s, k);
        else __syncthreads();
    }
    if (!a.hits) return;

    // ---- publish this CTA's list; the last CTA merges all of them
    Cand* mine = a.cand + (int64_t)blockIdx.x * k;
    for (int j = tid; j < k; j += kThreads) {
        Cand c;
        c.score = s.key[j];
        c.index = s.idx[j];
        c.payload = s.pay[j];
        mine[j] = c;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        // wraps to 0 when the last CTA arrives, ready for the next launch
        const unsigned int done = atomicInc(a.ticket, gridDim.x - 1);
        s.misc[1] = (done == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!s.misc[1]) return;
    __threadfence();

    topk_reset(s, 0);
    __syncthreads();
    const int64_t m = (int64_t)gridDim.x * k;
    const int round = kCap - k;
    for (int64_t r0 = 0; r0 < m; r0 += round) {
        for (int j = tid; j < round; j += kThreads) {
            const int64_t r = r0 + j;
            if (r < m) {
                const Cand* src = a.cand + r;
                const double sc = __ldcg(&src->score);
                const long long ix = __ldcg(reinterpret_cast<const long long*>(&src->index));
                const unsigned long long py =
                    __ldcg(reinterpret_cast<const unsigned long long*>(&src->payload));
                if (ix != kSentinelIndex) topk_offer(s, k, sc, (int64_t)ix, (uint64_t)py);
            }
        }
        topk_flush(s, k);
    }
    for (int j = tid; j < k; j += kThreads) {
        Hit h;
        h.index = s.idx[j];
        h.score = s.key[j];
        h.i1 = (uint32_t)(s.pay[j] & 0xffffffffu);
        h.i2 = (uint32_t)(s.pay[j] >> 32);
        const uint2 E = (h.index >= 0 && h.index < a.n) ? ecount2[h.index] : make_uint2(0, 0);
        h.e1 = E.x;
        h.e2 = E.y;
        h.p1 = P1;
        h.p2 = P2;
        a.hits[j] = h;
    }
}

}  // namespace

size_t scan_packed_smem(int chunk4)
{
    return (size_t)2 * chunk4 * sizeof(uint4) + (size_t)kCap * (8 + 8 + 8) +
           (size_t)kGroup * 2 * sizeof(uint32_t) + 4 * sizeof(int);
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
    const size_t smem = scan_packed_smem(a.chunk4);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
        kern<<<grid, kThreads, smem, stream>>>(a);
        return cudaGetLastError();
    };
    if (a.chunk4 <= kThreads) return run(scan_packed_kernel<1, 4>);
    if (a.chunk4 <= 2 * kThreads) return run(scan_packed_kernel<2, 2>);
    return run(scan_packed_kernel<4, 1>);
}

}  // namespace dbq
