// tc_scan.cu -- the exact loop of Section 2.3 (Ezhov et al. 2022) for many
// patients against one bit-packed database at once, on the tensor cores.
//
// For Q patients and N entries the intersections I_k(q, e) = |P_k(q) n E_k(e)|
// are dot products of 0/1 vectors over the V voxels: one dense contraction
// [Q x V] . [V x N] per segmentation.  The masks are stored as bits, which
// the tensor cores cannot read, so converter warps expand each K-slice of 256
// voxels of the patients' rows and of 224 entry rows into 4-bit E2M1 values
// (1.0 for a set bit, 0 otherwise; two voxels per byte) in the
// 128-byte-swizzled K-major layout of tcgen05 shared-memory operands, and one
// thread issues block-scaled tcgen05.mma (kind::mxf4, every UE8M0 scale 1.0;
// M = 128 patient rows -- the rows past Q are zero --, N = 224 entries,
// K = 64 per instruction) with binary32 accumulators in tensor memory.  An
// MMA instruction costs about the same for any N, so the entries, not the
// few patients, take the N side.  Every product is 0 or 1 and every partial
// sum an integer no larger than V <= 2^24, so the accumulators hold the
// exact counts.
//
// Voxel order inside a K-slice: a dot product does not depend on the order
// of its terms as long as both operands use the same one, so the expansion
// takes whatever order is cheapest: 16-byte chunk c of a row holds the 32
// voxels of bit word c, its 32-bit word j holds bits j, j + 4, ..., j + 28 of
// that word, one per nibble ((u >> j) & 0x11111111, shifted to the 1.0 code
// 0x2).  That is two integer instructions per 8 voxels.
//
//   * work units are (224-entry tile, segmentation), round-robin over one
//     persistent CTA per SM; each unit writes its own component of the
//     counts, so no unit waits for another;
//   * warp 1 (one thread, after allocating the 512 TMEM columns): TMA
//     producer.  Per 1024-voxel chunk of a unit it copies 128 bytes of every
//     entry row of the tile and of every patient row (3-D tensor maps over
//     [entry][plane][word], 128-byte swizzle) into one of two bit slots;
//     rows past the database's end and words past the plane's end arrive as
//     zeros.  Each row segment is one 128-byte request, which the memory
//     system serves far better than the 16- or 32-byte pieces that
//     per-thread loads of the tile's scattered rows make;
//   * warps 6-16 (converters): thread t < 224 expands entry row t of the
//     tile, thread 224 + r patient row r < Q; per K-slice each reads its
//     row's 32 bytes of bits from the bit slot, expands them into a 3-stage
//     ring of operand tiles and makes the stores visible to the tensor core
//     (fence.proxy.async); one lane per warp then arrives on the stage's full
//     barrier, and (after a chunk's fourth slice) on the bit slot's empty
//     barrier.  The patient rows past Q are cleared once;
//   * warp 0 (one thread): per K-slice four MMAs into the unit's 224
//     accumulator columns in one of two TMEM buffers (columns 0 and 256), so
//     the epilogue of a unit overlaps the next unit's MMAs; its commits free
//     the stage and, at the end of a unit, hand the buffer to the epilogue;
//   * warps 2-5 (epilogue, one TMEM lane quarter each, lane = patient row):
//     fill the scale columns (240-255 for A, 496-511 for B) with UE8M0 1.0
//     once, then tcgen05.ld the counts of 16 entries at a time and store them
//     as 64-byte rows of counts[plane][q][e].
// Shared memory: three operand stages of 44 KiB and two bit slots of
// 44 KiB.  Per 256-voxel slice about 114 KB pass through the shared-memory
// banks at 128 queries (TMA fills of the bits, the converters' reads of
// them, the expanded operand stores, the tensor core's operand reads), and
// the banks are busy about 92 % of the time: that traffic is the kernel's
// bound, not the tensor rate (the tensor pipe is busy about 46 %).  The
// mask sizes, binary64 scores and each patient's top-k follow in
// tc_select_kernel.  Every mbarrier wait is bounded; on a timeout the CTA
// records an error code in `status`, stops, lets its copies and MMAs finish
// and frees its TMEM.
#include "kernels.h"
#include "tcgen05.cuh"
#include "topk.cuh"

namespace dbq {
namespace {

constexpr int kTcQ = 128;                    // query rows of the MMA (M), zero-padded
constexpr int kTcE = 224;                    // entries per tile (MMA N)
constexpr int kTcMaxN = 128;                 // queries per launch
constexpr int kTcStages = 3;                 // operand stages, 44 KiB each
constexpr int kTcSlots = 2;                  // bit slots, 44 KiB each
constexpr int kTcConv = 352;                 // converter threads: 224 entry + 128 query rows
constexpr int kTcConvWarps = kTcConv / 32;
constexpr int kTcConv0 = 192;                // first converter thread (warps 0-5: MMA, TMA, epilogue)
constexpr int kTcThreads = kTcConv0 + kTcConv;
constexpr int kTcSliceWords = 8;             // 256 voxels per K-slice and row
constexpr int kTcChunkWords = 32;            // 1024 voxels (128 bytes) per row and bit slot
constexpr int kTcABytes = kTcQ * 128;        // query operand of a stage (and query bits of a slot)
constexpr int kTcBBytes = kTcE * 128;        // entry operand of a stage (and entry bits of a slot)
constexpr int kTcStageBytes = kTcABytes + kTcBBytes;
constexpr int kTcSlotBytes = kTcBBytes + kTcABytes;   // entry bits first, then query bits
constexpr uint32_t kTcBufCols = 256;         // TMEM columns between the two accumulators
constexpr uint32_t kTcScaleA = 240;          // TMEM columns of the unit scales
constexpr uint32_t kTcScaleB = 496;
constexpr uint32_t kUnitScales = 0x7F7F7F7Fu;   // four UE8M0 bytes of 2^0

static_assert(kTcE % 16 == 0 && kTcE <= 256 && kTcConv >= kTcE + kTcQ, "MMA N, converters");
static_assert(kTcScaleA >= kTcE && kTcScaleA + 16 <= kTcBufCols, "scale columns");
static_assert(kTcScaleB >= kTcBufCols + kTcE && kTcScaleB + 16 <= 512, "scale columns");
static_assert(kTcABytes % 1024 == 0 && kTcBBytes % 1024 == 0, "swizzle atoms");

// 1 KiB of alignment slack, the stages, the bit slots, the mbarriers (full
// and empty per stage and per slot, two accumulator pairs, the drain, the
// test stall), TMEM slot and abort flag.
constexpr int kTcBars = 2 * kTcStages + 2 * kTcSlots + 6;
size_t smem_bytes()
{
    return 1024 + (size_t)kTcStages * kTcStageBytes + (size_t)kTcSlots * kTcSlotBytes +
           kTcBars * 8 + 16;
}

__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr)
{
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

// 3-D tiled TMA load (x = word, y = plane, z = row), completion counted in
// bytes on `bar`.  x is a multiple of 32 words, 128 bytes.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}

__device__ __forceinline__ void st_global_v4(uint32_t* p, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d)
{
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}

__device__ __forceinline__ void umma_f4(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t sfa, uint32_t sfb,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
        " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], "
        "[%5], p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
        : "memory");
}

// Arrives on the mbarrier once the MMAs issued so far by this thread are done.
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

// 256 mask bits (eight words, voxel 32i + b = bit b of word i) -> one
// 128-byte operand row of E2M1 nibbles: chunk c (the 32 voxels of word c)
// goes to chunk position c ^ (row mod 8) of the row, the 128-byte swizzle.
__device__ __forceinline__ void expand_row(uint32_t row_base, int row, const uint4& lo,
                                           const uint4& hi)
{
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t u = w[c];
        st_shared_v4(row_base + (uint32_t)(((c ^ (row & 7)) & 7) << 4), (u << 1) & 0x22222222u,
                     u & 0x22222222u, (u >> 1) & 0x22222222u, (u >> 2) & 0x22222222u);
    }
}

// Byte offset of row `row` in a K-major 128-byte-swizzled column: 8-row
// groups of 1024 bytes, 128 bytes per row.
__device__ __forceinline__ uint32_t row_offset(int row)
{
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128);
}

__global__ void __launch_bounds__(kTcThreads, 1)
tc_scan_kernel(const __grid_constant__ CUtensorMap tm_db, const __grid_constant__ CUtensorMap tm_q,
               const TcScanArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* stages = base;                                  // kTcStages x (A | B)
    unsigned char* slots = stages + (size_t)kTcStages * kTcStageBytes;   // kTcSlots x (B | A) bits
    uint64_t* bars = reinterpret_cast<uint64_t*>(slots + (size_t)kTcSlots * kTcSlotBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kTcBars);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t ntiles = (a.n + kTcE - 1) / kTcE;
    const int64_t nunits = ntiles * 2;                             // (tile, plane)
    const int64_t my_units = nunits > blockIdx.x ? (nunits - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nk = (a.wp + kTcSliceWords - 1) / kTcSliceWords;       // K-slices per unit
    const int64_t nchunks = (a.wp + kTcChunkWords - 1) / kTcChunkWords;  // bit slots per unit

    const uint32_t full0 = smem_u32(bars);
    const uint32_t empty0 = smem_u32(bars + kTcStages);
    const uint32_t bfull0 = smem_u32(bars + 2 * kTcStages);
    const uint32_t bempty0 = smem_u32(bars + 2 * kTcStages + kTcSlots);
    const uint32_t acc_full0 = smem_u32(bars + 2 * kTcStages + 2 * kTcSlots);
    const uint32_t acc_free0 = acc_full0 + 16;
    const uint32_t drain = acc_full0 + 32;
    const uint32_t stall = acc_full0 + 40;                        // nothing ever arrives here

    // the query rows past nq stay zero in every stage: cleared once here
    for (int i = threadIdx.x; i < kTcStages * (kTcABytes / 16); i += blockDim.x) {
        const int st = i / (kTcABytes / 16), off = i % (kTcABytes / 16);
        const int row = ((off * 16) / 1024) * 8 + ((off * 16) % 1024) / 128;   // row of this 16 B
        if (row >= a.nq)
            *reinterpret_cast<uint4*>(stages + (size_t)st * kTcStageBytes + off * 16) =
                make_uint4(0, 0, 0, 0);
    }
    fence_proxy_async();
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(full0 + 8 * s, kTcConvWarps);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int s = 0; s < kTcSlots; ++s) {
            mbar_init(bfull0 + 8 * s, 1);
            mbar_init(bempty0 + 8 * s, kTcConvWarps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full0 + 8 * b, 1);
            mbar_init(acc_free0 + 8 * b, 128);
        }
        mbar_init(drain, 1);
        mbar_init(stall, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (warp >= 2 && warp < 6) {
        // unit scales for both operands, every lane of this warp's quarter
        const uint32_t lanes = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, "
            "%1, %1, %1, %1, %1, %1, %1};" ::"r"(lanes + kTcScaleA),
            "r"(kUnitScales)
            : "memory");
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, "
            "%1, %1, %1, %1, %1, %1, %1};" ::"r"(lanes + kTcScaleB),
            "r"(kUnitScales)
            : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0) {
        if (lane == 0) {
            // block-scaled descriptor: A and B E2M1 (MXF4 format 1), K-major,
            // UE8M0 scales, N = 224 entries, M = 128 query rows, K = 64
            const uint32_t idesc = (1u << 7) | (1u << 10) | ((uint32_t)(kTcE >> 3) << 17) |
                                   (1u << 23) | ((uint32_t)(kTcQ >> 4) << 24);
            int s = 0;
            uint32_t phase = 0;
            bool ok = true;
            if (a.stall_ns && !mbar_wait_for(stall, 0, abort_flag, a.stall_ns)) {
                a.status[0] = 5;           // the test stall ran out, as it must
                ok = false;
            }
            const uint64_t desc0 = sw128_desc(smem_u32(stages));
            const uint64_t b_off = (uint64_t)(kTcABytes >> 4);
            uint64_t sdesc = desc0;
            for (int64_t u = 0; u < my_units && ok; ++u) {
                const int buf = (int)(u & 1);
                if (!mbar_wait(acc_free0 + 8 * buf, (uint32_t)(((u >> 1) & 1) ^ 1), abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)buf * kTcBufCols;
                for (int64_t kc = 0; kc < nk; ++kc) {
                    if (!mbar_wait(full0 + 8 * s, phase, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)   // 64 voxels = 32 bytes per row each
                        umma_f4(d_tmem, sdesc + (uint64_t)(2 * kk), sdesc + b_off + (uint64_t)(2 * kk),
                                idesc, tmem + kTcScaleA, tmem + kTcScaleB,
                                (kc > 0 || kk > 0) ? 1u : 0u);
                    umma_commit(empty0 + 8 * s);
                    sdesc += kTcStageBytes >> 4;
                    if (++s == kTcStages) {
                        s = 0;
                        phase ^= 1u;
                        sdesc = desc0;
                    }
                }
                if (ok) umma_commit(acc_full0 + 8 * buf);
            }
            if (!ok) {
                if (a.status[0] == 0) a.status[0] = 2;
                *abort_flag = 1;
            }
            umma_commit(drain);
            if (!mbar_wait(drain, 0, nullptr)) a.status[0] = 3;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // TMA producer: per unit and 1024-voxel chunk, the 128-byte row
            // segments of the tile's entries and of the patients
            int slot = 0;
            uint32_t phase = 0;
            bool issued[kTcSlots] = {};
            uint32_t issued_parity[kTcSlots] = {};
            const uint32_t slot0 = smem_u32(slots);
            const uint32_t bytes = (uint32_t)(kTcE + a.nq) * 128u;
            bool ok = true;
            for (int64_t u = 0; u < my_units && ok; ++u) {
                const int64_t unit = blockIdx.x + u * gridDim.x;
                const int plane = (int)(unit & 1);
                const int e0 = (int)((unit >> 1) * kTcE);
                for (int64_t j = 0; j < nchunks; ++j) {
                    if (!mbar_wait(bempty0 + 8 * slot, phase ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = slot0 + (uint32_t)(slot * kTcSlotBytes);
                    mbar_arrive_expect_tx(bfull0 + 8 * slot, bytes);
                    tma_load_3d(dst, &tm_db, bfull0 + 8 * slot, (int)(j * kTcChunkWords), plane, e0);
                    tma_load_3d(dst + kTcBBytes, &tm_q, bfull0 + 8 * slot, (int)(j * kTcChunkWords),
                                plane, 0);
                    issued[slot] = true;
                    issued_parity[slot] = phase;
                    if (++slot == kTcSlots) {
                        slot = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                if (a.status[0] == 0) a.status[0] = 6;
                *abort_flag = 1;
            }
            // no copy may still be writing shared memory when the CTA exits
            for (int sl = 0; sl < kTcSlots; ++sl)
                if (issued[sl] && !mbar_wait(bfull0 + 8 * sl, issued_parity[sl], nullptr))
                    a.status[0] = 7;
        }
    } else if (warp >= 2 && warp < 6) {
        // lane = query row; columns = the unit's 224 entries
        const int quarter = warp & 3;
        const int q = quarter * 32 + lane;
        for (int64_t u = 0; u < my_units; ++u) {
            const int buf = (int)(u & 1);
            if (!mbar_wait(acc_full0 + 8 * buf, (uint32_t)((u >> 1) & 1), abort_flag)) {
                if (a.status[0] == 0) a.status[0] = 4;
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int64_t unit = blockIdx.x + u * gridDim.x;
            const int64_t e0 = (unit >> 1) * kTcE;
            const int plane = (int)(unit & 1);
            const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)buf * kTcBufCols;
            for (int c0 = 0; c0 < kTcE; c0 += 16) {
                uint32_t r[16];
                tmem_ld16(lane_base + c0, r);
                tmem_wait_ld();
                if (q < a.nq) {
                    uint32_t* row = a.counts + ((int64_t)plane * a.nq + q) * a.stride;
                    uint32_t v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = (uint32_t)__uint_as_float(r[j]);   // exact
                    const int64_t e = e0 + c0;
                    if (e + 16 <= a.n) {
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            st_global_v4(row + e + j, v[j], v[j + 1], v[j + 2], v[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (e + j < a.n) row[e + j] = v[j];
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acc_free0 + 8 * buf);
        }
    } else if (warp >= kTcConv0 / 32) {
        // converters: thread ct < 224 expands entry row ct of the tile, thread
        // 224 + r query row r (r < nq)
        const int ct = threadIdx.x - kTcConv0;
        const bool is_b = ct < kTcE;
        const int row = is_b ? ct : ct - kTcE;
        const bool active = is_b || row < a.nq;
        const int srow = active ? row : 0;
        const uint32_t dst = (is_b ? (uint32_t)kTcABytes : 0u) + row_offset(srow);
        const uint32_t src = smem_u32(slots) + (is_b ? 0u : (uint32_t)kTcBBytes) + (uint32_t)(srow * 128);
        const uint32_t stage0 = smem_u32(stages);
        int s = 0, slot = 0;
        uint32_t phase = 0, bphase = 0;
        bool ok = true;
        for (int64_t u = 0; u < my_units && ok; ++u) {
            for (int64_t kc = 0; kc < nk; ++kc) {
                const int c4 = (int)(kc & 3);      // slice within the bit slot's chunk
                int r = 1;
                if (c4 == 0) {
                    if (lane == 0) r = mbar_wait(bfull0 + 8 * slot, bphase, abort_flag);
                    r = __shfl_sync(0xffffffffu, r, 0);
                    if (!r) {
                        ok = false;
                        break;
                    }
                }
                uint4 lo = make_uint4(0, 0, 0, 0), hi = lo;
                if (active) {   // the slot holds the row's 128 bytes swizzled like the operands
                    const uint32_t sb = src + (uint32_t)(slot * kTcSlotBytes);
                    lo = ld_shared_v4(sb + (uint32_t)((((2 * c4) ^ (srow & 7)) & 7) << 4));
                    hi = ld_shared_v4(sb + (uint32_t)((((2 * c4 + 1) ^ (srow & 7)) & 7) << 4));
                }
                if (lane == 0) r = mbar_wait(empty0 + 8 * s, phase ^ 1u, abort_flag);
                r = __shfl_sync(0xffffffffu, r, 0);
                if (!r) {
                    ok = false;
                    break;
                }
                if (active) expand_row(stage0 + (uint32_t)(s * kTcStageBytes) + dst, row, lo, hi);
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(full0 + 8 * s);
                if (++s == kTcStages) {
                    s = 0;
                    phase ^= 1u;
                }
                if (c4 == 3 || kc == nk - 1) {   // the chunk's bits are no longer needed
                    if (lane == 0) mbar_arrive(bempty0 + 8 * slot);
                    if (++slot == kTcSlots) {
                        slot = 0;
                        bphase ^= 1u;
                    }
                }
            }
        }
        if (!ok && lane == 0) {
            if (a.status[0] == 0) a.status[0] = 1;
            *abort_flag = 1;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem)
                     : "memory");
    }
}

// Scores and top-k of one patient (one CTA per patient) from its counts:
// the same binary64 Dice scores, keys and order as the fused scans.
__global__ void __launch_bounds__(1024, 1)
tc_select_kernel(const QueryTask* __restrict__ tasks, int task0, int nq,
                 const uint32_t* __restrict__ counts, int64_t n, int64_t stride)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TopK tk;
    topk_carve(tk, smem_raw);
    const QueryTask& t = tasks[task0 + blockIdx.x];
    const int k = t.k;
    const uint32_t P1 = t.pcount[0], P2 = t.pcount[1];
    const uint2* ecount2 = reinterpret_cast<const uint2*>(t.ecount);
    const uint32_t* row1 = counts + (int64_t)blockIdx.x * stride;
    const uint32_t* row2 = counts + ((int64_t)nq + blockIdx.x) * stride;
    topk_init(tk);
    for (int64_t b0 = 0; b0 < n; b0 += blockDim.x) {
        const int64_t e = b0 + threadIdx.x;
        if (e < n) {
            const uint32_t I1 = row1[e], I2 = row2[e];
            const uint2 E = ecount2[e];
            topk_offer_counts(tk, k, I1, I2, E.x, E.y, P1, P2, e);
        }
        __syncthreads();
        // room for another round of offers
        if (tk.misc[0] > kTopkCap - k - (int)blockDim.x) topk_flush(tk, k);
    }
    topk_flush(tk, k);
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
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

}  // namespace

int tc_scan_max_queries() { return kTcMaxN; }

int64_t tc_counts_stride(int64_t n) { return (n + 3) / 4 * 4; }

// 3-D map [rows][2 planes][wp words] of uint32 with a box of 32 words x 1
// plane x box_rows rows, 128-byte swizzle; out-of-range rows and words read
// as zeros.
static bool make_bits_map(CUtensorMap* m, const void* base, int64_t wp, int64_t rows, int box_rows)
{
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)wp, 2, (cuuint64_t)rows};
    const cuuint64_t strides[2] = {(cuuint64_t)wp * 4, (cuuint64_t)wp * 8};
    const cuuint32_t box[3] = {(cuuint32_t)kTcChunkWords, 1, (cuuint32_t)box_rows};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<void*>(base), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_tc_scan(const TcScanArgs& a, int grid, cudaStream_t stream)
{
    if (a.nq < 1 || a.nq > kTcMaxN || a.n < 1 || a.n > INT32_MAX || a.wp < kTcChunkWords ||
        a.wp % 4 != 0 || a.stride < a.n || a.stride % 4 != 0 ||
        (reinterpret_cast<uintptr_t>(a.planes) & 15) || (reinterpret_cast<uintptr_t>(a.qplanes) & 15) ||
        (reinterpret_cast<uintptr_t>(a.counts) & 15))
        return cudaErrorInvalidValue;
    CUtensorMap tm_db, tm_q;
    if (!make_bits_map(&tm_db, a.planes, a.wp, a.n, kTcE) ||
        !make_bits_map(&tm_q, a.qplanes, a.wp, a.nq, a.nq))
        return cudaErrorInvalidValue;
    const size_t smem = smem_bytes();
    cudaError_t err = cudaFuncSetAttribute(tc_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    const int64_t nunits = (a.n + kTcE - 1) / kTcE * 2;
    if (grid > nunits) grid = (int)nunits;
    if (grid < 1) grid = 1;
    tc_scan_kernel<<<grid, kTcThreads, smem, stream>>>(tm_db, tm_q, a);
    return cudaGetLastError();
}

int64_t tc_scan_min_words() { return kTcChunkWords; }

cudaError_t launch_tc_select(const QueryTask* tasks, int task0, int nq, const uint32_t* counts,
                             int64_t n, int64_t stride, cudaStream_t stream)
{
    if (nq < 1 || n < 1 || stride < n) return cudaErrorInvalidValue;
    const size_t smem = topk_smem_bytes();
    cudaError_t err = cudaFuncSetAttribute(tc_select_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    tc_select_kernel<<<nq, 1024, smem, stream>>>(tasks, task0, nq, counts, n, stride);
    return cudaGetLastError();
}

}  // namespace dbq
