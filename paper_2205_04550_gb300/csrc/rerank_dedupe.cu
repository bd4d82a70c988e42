// rerank_dedupe.cu -- exact re-ranking of a batch's prefilter candidates that
// reads each distinct candidate entry once.
//
// The queries of one embedding batch pick overlapping candidates (on 256
// queries x 512 candidates of 100,000 entries of 128^3 voxels, 54 % of the
// (query, candidate) pairs are distinct entries), and the per-query
// re-ranking of rerank.cu reads every pair's entry from HBM.  Here:
//
//   1. the pairs are sorted by entry (a counting sort: histogram, prefix sum,
//      scatter), giving the distinct entries in ascending order and each
//      entry's run of pairs;
//   2. the planes are cut into slices of 32 16-byte words.  A CTA owns one
//      slice of one plane: it holds that slice of every query's patient plane
//      in shared memory (nq x 512 bytes), then streams the same slice of every
//      distinct entry once and intersects it with the patient slice of each
//      query that picked the entry.  A slice count is at most 4,096 bits, so
//      it is written as 16 bits per pair and slice;
//   3. the slice counts are summed per pair and plane;
//   4. a CTA per query scores its candidates exactly (binary64 Dice at both
//      thresholds, summed, Section 2.3 of Ezhov et al. 2022) and keeps the
//      top-k with the shared top-k code -- the hits of rerank.cu, bit for bit,
//      because the counts are exact and the ranking is a total order.
//
// A tumour fills a small part of the grid, so most queries' patient slices
// are empty: those pairs intersect nothing in the slice and only their zero
// count is written, which leaves the warps mostly streaming the entries'
// pieces (every word of every distinct entry is still read).  The histogram
// returns to zero in the scatter, so only its allocation clears it.
#include "kernels.h"
#include "topk.cuh"

namespace dbq {
namespace {

constexpr int kSliceW = 32;          // 16-byte words per plane slice (one per lane)
constexpr int kCountThreads = 1024;
constexpr int kEntryBatch = 6;       // entries a warp loads before it counts them
constexpr int kScanThreads2 = 1024;
constexpr int kScanPer = 4;          // histogram bins per thread per tile
constexpr int kScanTile = kScanThreads2 * kScanPer;
constexpr int kReduceThreads = 256;
constexpr int kSelectThreads = 1024;

// popc(a & b) over four words (at most 128).
__device__ __forceinline__ uint32_t and_popc4(uint4 a, uint4 b)
{
    return __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
}

// hist[e] += pairs naming entry e.
__global__ void rr_hist_kernel(const int32_t* __restrict__ cand, int64_t npairs,
                               uint32_t* __restrict__ hist)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs;
         p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[cand[p]], 1u);
}

// Block-exclusive prefix of (pairs, distinct entries) over the threads.
__device__ __forceinline__ void block_scan2(uint32_t& a, uint32_t& b, uint32_t* sa, uint32_t* sb,
                                            uint32_t& tot_a, uint32_t& tot_b)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, ia, o);
        const uint32_t y = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += x;
            ib += y;
        }
    }
    if (lane == 31) {
        sa[warp] = ia;
        sb[warp] = ib;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t x = lane < nw ? sa[lane] : 0u, y = lane < nw ? sb[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
            const uint32_t v = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) {
                x += u;
                y += v;
            }
        }
        if (lane < nw) {
            sa[lane] = x;
            sb[lane] = y;
        }
    }
    __syncthreads();
    tot_a = sa[(blockDim.x >> 5) - 1];
    tot_b = sb[(blockDim.x >> 5) - 1];
    const uint32_t wa = warp ? sa[warp - 1] : 0u, wb = warp ? sb[warp - 1] : 0u;
    a = wa + ia - a;
    b = wb + ib - b;
    __syncthreads();   // sa / sb are reused by the next call
}

// Per tile of kScanTile bins: (pairs, distinct entries).
__global__ void __launch_bounds__(kScanThreads2)
rr_tile_sums_kernel(const uint32_t* __restrict__ hist, int64_t n, uint2* __restrict__ tiles)
{
    __shared__ uint32_t sa[32], sb[32];
    const int64_t e0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    uint32_t s = 0, z = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const uint32_t h = e0 + i < n ? hist[e0 + i] : 0u;
        s += h;
        z += h ? 1u : 0u;
    }
    uint32_t ta, tb;
    block_scan2(s, z, sa, sb, ta, tb);
    if (threadIdx.x == 0) tiles[blockIdx.x] = make_uint2(ta, tb);
}

// start[e] = pairs of entries below e (start[n] = all pairs); the distinct
// entries ascending, uniq[0 .. *nuniq), with their first pair ubeg[u]
// (ubeg[*nuniq] = all pairs).
__global__ void __launch_bounds__(kScanThreads2)
rr_scan_kernel(const uint32_t* __restrict__ hist, int64_t n, const uint2* __restrict__ tiles,
               uint32_t* __restrict__ start, int32_t* __restrict__ uniq,
               uint32_t* __restrict__ ubeg, uint32_t* __restrict__ nuniq)
{
    __shared__ uint32_t sa[32], sb[32];
    __shared__ uint32_t base_a, base_b;
    if (threadIdx.x < 32) {
        uint32_t x = 0, y = 0;
        for (int t = threadIdx.x; t < (int)blockIdx.x; t += 32) {
            const uint2 v = tiles[t];
            x += v.x;
            y += v.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if (threadIdx.x == 0) {
            base_a = x;
            base_b = y;
        }
    }
    __syncthreads();
    const int64_t e0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    uint32_t h[kScanPer];
    uint32_t s = 0, z = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        h[i] = e0 + i < n ? hist[e0 + i] : 0u;
        s += h[i];
        z += h[i] ? 1u : 0u;
    }
    uint32_t ta, tb;
    block_scan2(s, z, sa, sb, ta, tb);
    uint32_t run = base_a + s, urun = base_b + z;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (e0 + i < n) {
            start[e0 + i] = run;
            if (h[i]) {
                uniq[urun] = (int32_t)(e0 + i);
                ubeg[urun] = run;
                ++urun;
            }
            run += h[i];
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        start[n] = base_a + ta;
        ubeg[base_b + tb] = base_a + ta;
        *nuniq = base_b + tb;
    }
}

// Pair p (query p / c) goes to position start[cand[p]] + slot; hist returns
// to zero.  qof[pos] = its query, posof[p] = pos.
__global__ void rr_scatter_kernel(const int32_t* __restrict__ cand, int64_t npairs, int c,
                                  const uint32_t* __restrict__ start, uint32_t* __restrict__ hist,
                                  uint16_t* __restrict__ qof, uint32_t* __restrict__ posof)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = cand[p];
        const uint32_t pos = start[e] + atomicSub(&hist[e], 1u) - 1u;
        qof[pos] = (uint16_t)(p / c);
        posof[p] = pos;
    }
}

// Slice counts.  grid (2 * nslice, ysplit): CTA x owns words [32 s, 32 s + 32)
// of plane x / nslice (s = x % nslice) and the y-th part of the distinct
// entries; each warp takes a contiguous run of them, kEntryBatch at a time:
// it loads their pieces (one 16-byte word per lane, 512 bytes per entry),
// then intersects each with the patient slice of every query in the entry's
// run of pairs.  Results go to partial[x][pos], 16 bits, written 32
// positions at a time.
__global__ void __launch_bounds__(kCountThreads, 1)
rr_count_kernel(const uint4* __restrict__ planes, int wp4, const uint4* __restrict__ patients,
                int nq, const int32_t* __restrict__ uniq, const uint32_t* __restrict__ ubeg,
                const uint32_t* __restrict__ nuniq, const uint16_t* __restrict__ qof, int nslice,
                int64_t pstride, uint16_t* __restrict__ partial)
{
    // [nq][kSliceW] patient slices, [warps][32][32] staging bytes, [nq] flags
    extern __shared__ uint4 spat[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t* stage = reinterpret_cast<uint8_t*>(spat + nq * kSliceW) + warp * 1024;
    uint8_t* nonzero = reinterpret_cast<uint8_t*>(spat + nq * kSliceW) +
                       (kCountThreads / 32) * 1024;
    const int x = blockIdx.x;
    const int plane = x / nslice;
    const int w0 = (x - plane * nslice) * kSliceW;
    // a warp loads whole slices (kSliceW = 32 lanes, blockDim a multiple of
    // 32) and flags the queries whose slice has a set bit: a pair whose
    // query's slice is empty intersects nothing here, so only its zero count
    // is written
    for (int i = threadIdx.x; i < nq * kSliceW; i += blockDim.x) {
        const int q = i / kSliceW, w = w0 + i % kSliceW;
        const uint4 v =
            w < wp4 ? patients[((int64_t)q * 2 + plane) * wp4 + w] : make_uint4(0, 0, 0, 0);
        spat[i] = v;
        const bool any = __any_sync(0xffffffffu, (v.x | v.y | v.z | v.w) != 0u);
        if (lane == 0) nonzero[q] = any ? 1 : 0;
    }
    __syncthreads();
    // entry indices are int32, so the distinct entries number below 2^31
    const int nu = (int)*nuniq;
    const int c0 = (int)((int64_t)nu * blockIdx.y / gridDim.y);
    const int c1 = (int)((int64_t)nu * (blockIdx.y + 1) / gridDim.y);
    const int nwarps = blockDim.x >> 5;
    const int per = (c1 - c0 + nwarps - 1) / nwarps;
    const int u_begin = c0 + per * warp;
    const int u_end = c1 < u_begin + per ? c1 : u_begin + per;
    const bool live = w0 + lane < wp4;
    const uint4* src = planes + (int64_t)plane * wp4 + w0 + lane;
    const int64_t estride = 2 * (int64_t)wp4;
    uint16_t* out = partial + (int64_t)x * pstride;
    // batches of kEntryBatch entries: the pieces of a batch are loaded
    // together (kEntryBatch x 512 bytes in flight per warp), then counted.
    // The next batch's entry ids and pair bounds are loaded while this one
    // is counted, so a batch waits on one memory latency, not two.
    auto batch_len = [&](int u) { return u_end - u < kEntryBatch ? u_end - u : kEntryBatch; };
    uint32_t bn = 0;   // lanes 0..nb: the first pair of entry u0 + lane (lane nb: the end)
    int32_t en = 0;    // lanes 0..nb-1: the entries
    if (u_begin < u_end) {
        const int nb = batch_len(u_begin);
        bn = ubeg[u_begin + (lane < nb ? lane : nb)];
        en = uniq[u_begin + (lane < nb - 1 ? lane : nb - 1)];
    }
    for (int u0 = u_begin; u0 < u_end; u0 += kEntryBatch) {
        const int nb = batch_len(u0);
        const uint32_t b = bn;
        const int32_t e = en;
        const int u1 = u0 + kEntryBatch;
        if (u1 < u_end) {
            const int nb1 = batch_len(u1);
            bn = ubeg[u1 + (lane < nb1 ? lane : nb1)];
            en = uniq[u1 + (lane < nb1 - 1 ? lane : nb1 - 1)];
        }
        uint4 ev[kEntryBatch];
#pragma unroll
        for (int j = 0; j < kEntryBatch; ++j) {
            const int32_t ej = __shfl_sync(0xffffffffu, e, j);
            ev[j] = make_uint4(0, 0, 0, 0);
            if (j < nb && live) ev[j] = ld_stream(src + (int64_t)ej * estride);
        }
        const uint32_t s_first = __shfl_sync(0xffffffffu, b, 0);
        const uint32_t s_last = __shfl_sync(0xffffffffu, b, nb);
        // positions in windows of 32: lane i of the warp holds the patient
        // slice offset of position wbase + i; each lane's partial count of
        // position wbase + i goes to stage[i][lane] (at most 128: a byte),
        // and lane i sums row i
        for (uint32_t wbase = s_first; wbase < s_last; wbase += 32u) {
            const int wn = s_last - wbase < 32u ? (int)(s_last - wbase) : 32;
            const uint32_t q = lane < wn ? (uint32_t)qof[wbase + lane] : 0u;
            const bool counted = lane < wn && nonzero[q];
            const uint32_t qoff = q * (uint32_t)kSliceW;
            // positions of the window whose query's slice is not empty
            const unsigned act = __ballot_sync(0xffffffffu, counted);
#pragma unroll
            for (int j = 0; j < kEntryBatch; ++j) {
                if (j < nb) {
                    const int p0 = (int)__shfl_sync(0xffffffffu, b, j) - (int)wbase;
                    const int p1 = (int)__shfl_sync(0xffffffffu, b, j + 1) - (int)wbase;
                    const int i0 = p0 > 0 ? p0 : 0;
                    const int i1 = p1 < wn ? p1 : wn;
                    unsigned m = 0u;
                    if (i0 < i1)   // bits [i0, i1); i0 < 32
                        m = act & (i1 >= 32 ? 0xffffffffu : (1u << i1) - 1u) & ~((1u << i0) - 1u);
                    while (m) {
                        const int ia = __ffs(m) - 1;
                        m &= m - 1u;
                        const uint4 pa = spat[__shfl_sync(0xffffffffu, qoff, ia) + lane];
                        if (m) {   // two independent chains
                            const int ib = __ffs(m) - 1;
                            m &= m - 1u;
                            const uint4 pb = spat[__shfl_sync(0xffffffffu, qoff, ib) + lane];
                            stage[ib * 32 + lane] = (uint8_t)and_popc4(ev[j], pb);
                        }
                        stage[ia * 32 + lane] = (uint8_t)and_popc4(ev[j], pa);
                    }
                }
            }
            __syncwarp();
            if (lane < wn && !counted) out[wbase + lane] = 0;
            if (counted) {
                const uint4* row = reinterpret_cast<const uint4*>(stage + lane * 32);
                const uint4 r0 = row[0], r1 = row[1];
                uint32_t t = 0;
                t = __dp4a(r0.x, 0x01010101u, t);
                t = __dp4a(r0.y, 0x01010101u, t);
                t = __dp4a(r0.z, 0x01010101u, t);
                t = __dp4a(r0.w, 0x01010101u, t);
                t = __dp4a(r1.x, 0x01010101u, t);
                t = __dp4a(r1.y, 0x01010101u, t);
                t = __dp4a(r1.z, 0x01010101u, t);
                t = __dp4a(r1.w, 0x01010101u, t);
                out[wbase + lane] = (uint16_t)t;
            }
            __syncwarp();
        }
    }
}

// cnt[plane][pos] = sum over the plane's slices.  grid (ceil(pstride / 2 /
// kReduceThreads), 2); thread i sums positions 2i and 2i + 1 (pstride even).
__global__ void __launch_bounds__(kReduceThreads)
rr_reduce_kernel(const uint16_t* __restrict__ partial, int nslice, int64_t pstride,
                 int64_t npairs, uint32_t* __restrict__ cnt)
{
    const int plane = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * i >= npairs) return;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(partial + (int64_t)plane * nslice * pstride) + i;
    const int64_t stride = pstride / 2;
    uint32_t lo = 0, hi = 0;
    int s = 0;
    for (; s + 8 <= nslice; s += 8) {
        uint32_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcs(src + (int64_t)(s + u) * stride);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            lo += v[u] & 0xffffu;
            hi += v[u] >> 16;
        }
    }
    for (; s < nslice; ++s) {
        const uint32_t v = __ldcs(src + (int64_t)s * stride);
        lo += v & 0xffffu;
        hi += v >> 16;
    }
    cnt[plane * npairs + 2 * i] = lo;
    if (2 * i + 1 < npairs) cnt[plane * npairs + 2 * i + 1] = hi;
}

// One CTA per query: exact scores of its c candidates from the summed
// counts, top-k, hits.
__global__ void __launch_bounds__(kSelectThreads, 1)
rr_select_kernel(const RerankArgs a, const uint32_t* __restrict__ posof,
                 const uint32_t* __restrict__ cnt, int64_t npairs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TopK tk;
    topk_carve(tk, smem_raw);
    const int q = blockIdx.x;
    const uint32_t P1 = a.pcounts[2 * q], P2 = a.pcounts[2 * q + 1];
    const uint2* ecount2 = reinterpret_cast<const uint2*>(a.ecount);
    topk_init(tk);
    for (int i0 = 0; i0 < a.c; i0 += blockDim.x) {
        const int i = i0 + (int)threadIdx.x;
        if (i < a.c) {
            const int64_t p = (int64_t)q * a.c + i;
            const uint32_t pos = posof[p];
            const int64_t e = a.cand[p];
            const uint2 E = ecount2[e];
            topk_offer_counts(tk, a.k, cnt[pos], cnt[npairs + pos], E.x, E.y, P1, P2, e);
        }
        topk_flush(tk, a.k);
    }
    for (int j = threadIdx.x; j < a.k; j += blockDim.x) {
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

}  // namespace

int rerank_dedupe_slices(int wp4) { return (wp4 + kSliceW - 1) / kSliceW; }

int64_t rerank_dedupe_pstride(int64_t npairs) { return (npairs + 63) / 64 * 64; }

int64_t rerank_dedupe_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

cudaError_t launch_rerank_dedupe(const RerankArgs& a, const RerankDedupeWork& w,
                                 cudaStream_t stream)
{
    if (a.nq < 1 || a.nq > kRerankDedupeMaxQ || a.c < 1 || a.c > kSelectThreads || a.k < 1 ||
        a.k > a.c || a.sup_lists || a.n < 1 || a.wp4 < 1)
        return cudaErrorInvalidValue;
    const int64_t npairs = (int64_t)a.nq * a.c;
    const int nslice = rerank_dedupe_slices(a.wp4);
    const int64_t pstride = rerank_dedupe_pstride(npairs);
    if (w.partial_elems < (int64_t)2 * nslice * pstride) return cudaErrorInvalidValue;
    // attributes first: once the histogram is built, every launch must follow
    // (the scatter returns it to zero)
    const size_t csmem =
        (size_t)a.nq * kSliceW * sizeof(uint4) + (kCountThreads / 32) * 1024 + a.nq;
    const size_t ssmem = topk_smem_bytes();
    cudaError_t err = cudaFuncSetAttribute(rr_count_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(rr_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)ssmem);
    if (err != cudaSuccess) return err;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int pgrid = (int)std::min<int64_t>((npairs + 255) / 256, (int64_t)sms * 8);
    rr_hist_kernel<<<pgrid, 256, 0, stream>>>(a.cand, npairs, w.hist);
    const int tiles = (int)rerank_dedupe_tiles(a.n);
    rr_tile_sums_kernel<<<tiles, kScanThreads2, 0, stream>>>(w.hist, a.n, w.tiles);
    rr_scan_kernel<<<tiles, kScanThreads2, 0, stream>>>(w.hist, a.n, w.tiles, w.start, w.uniq,
                                                         w.ubeg, w.nuniq);
    rr_scatter_kernel<<<pgrid, 256, 0, stream>>>(a.cand, npairs, a.c, w.start, w.hist, w.qof,
                                                  w.posof);
    const int gx = 2 * nslice;
    const int gy = gx >= 2 * sms ? 1 : (2 * sms + gx - 1) / gx;
    rr_count_kernel<<<dim3(gx, gy), kCountThreads, csmem, stream>>>(
        a.planes, a.wp4, a.patients, a.nq, w.uniq, w.ubeg, w.nuniq, w.qof, nslice, pstride,
        w.partial);
    const int rx = (int)((pstride / 2 + kReduceThreads - 1) / kReduceThreads);
    rr_reduce_kernel<<<dim3(rx, 2), kReduceThreads, 0, stream>>>(w.partial, nslice, pstride,
                                                                 npairs, w.cnt);
    rr_select_kernel<<<a.nq, kSelectThreads, ssmem, stream>>>(a, w.posof, w.cnt, npairs);
    return cudaGetLastError();
}

}  // namespace dbq
