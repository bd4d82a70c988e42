// noalloc.cu -- db_scan_packed_noalloc: the bit-packed exact query for callers
// that cannot allocate device memory.
//
// Who cannot allocate: a serving process whose memory pool has already
// reserved the whole GPU (a cudaMalloc there either fails or competes with
// the pool), code that runs on a request path where a device allocation's
// implicit synchronisation is not acceptable, and hosts that embed this
// library as a plug-in and forbid it to own device memory.  The handle API
// (db_create and the calls after it) allocates the database and a query
// workspace, so it does not serve them.  This entry point takes every input
// and output from the caller and keeps its only scratch -- the per-CTA
// candidate lists and the arrival ticket of the fused scan -- in one
// file-scope device array, so it allocates nothing itself.
//
// Costs and limits:
//   * the array (kScratchBytes + 256 bytes = 512.25 KiB) exists on every GPU
//     that loads the library, until the process exits;
//   * k <= 64 hits per call, and at most 256 SMs on the device;
//   * every call shares the array: calls whose work overlaps on the GPU (two
//     streams, or two host threads, with no ordering between them) race on it
//     and can return wrong hits.  The ticket is cleared on the caller's
//     stream before each launch; the candidate lists are fully rewritten by
//     every launch and need no clearing;
//   * every call made outside stream capture looks up the array's device
//     address (cudaGetSymbolAddress) for the current device and caches it;
//     a call made while its stream is being captured uses that cached
//     address, so the first call on a device must come before any capture.
//     Looking the address up again on every uncaptured call keeps it valid
//     after the primary context has been torn down and created again (a
//     cudaDeviceReset reloads the module at a new address).
#include <mutex>

#include "dbq.h"
#include "kernels.h"

namespace {

constexpr int kMaxNoallocK = 64;        // hits per call
constexpr int kMaxNoallocCtas = 256;    // one CTA per SM
constexpr size_t kScratchBytes = (size_t)kMaxNoallocK * kMaxNoallocCtas * sizeof(dbq::Cand);

// [0, kScratchBytes): candidate lists; [kScratchBytes, +256): ticket.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes + 256];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

int noalloc_fail(int code, const char* msg) { return dbq::record_error(code, msg); }

}  // namespace

extern "C" int db_scan_packed_noalloc(const uint32_t* planes, const uint32_t* sizes, int64_t n,
                                      int64_t stride_words, const uint32_t* patient_planes,
                                      const uint32_t* patient_sizes, int k, dbq_hit* hits,
                                      void* stream)
{
    if (!planes || !sizes || !patient_planes || !patient_sizes || !hits)
        return noalloc_fail(DBQ_EINVAL, "NULL pointer argument");
    if (n < 1) return noalloc_fail(DBQ_EINVAL, "n must be >= 1");
    if (stride_words < 4 || stride_words % 4 != 0 || stride_words / 4 > INT32_MAX)
        return noalloc_fail(DBQ_EINVAL, "stride_words must be a positive multiple of 4");
    if ((reinterpret_cast<uintptr_t>(planes) | reinterpret_cast<uintptr_t>(patient_planes)) % 16 ||
        reinterpret_cast<uintptr_t>(sizes) % 8 || reinterpret_cast<uintptr_t>(hits) % 8)
        return noalloc_fail(DBQ_EINVAL, "planes must be 16-byte and sizes/hits 8-byte aligned");
    if (k < 1 || k > kMaxNoallocK || k > n)
        return noalloc_fail(DBQ_ERANGE, "k must be in [1, min(n, 64)]");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(DBQ_ECUDA, "no usable current device");
    const int grid = dbq::scan_packed_grid(dev);
    if (grid > kMaxNoallocCtas)
        return noalloc_fail(DBQ_ERANGE, "device has more SMs than the scratch array serves");

    // The device address of the scratch array: looked up (and cached per
    // device) by every call outside stream capture, taken from the cache
    // during capture.
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &capture) != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(DBQ_ECUDA, "cannot query the stream's capture status");
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (capture == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (err != cudaSuccess || !p) {
                cudaGetLastError();
                return noalloc_fail(DBQ_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
            }
            g_scratch_addr[dev] = p;
        } else if (!g_scratch_addr[dev]) {
            return noalloc_fail(DBQ_ESTATE,
                                "the first call on a device must come before any stream capture");
        }
        scratch = g_scratch_addr[dev];
    }
    unsigned char* base = static_cast<unsigned char*>(scratch);
    unsigned int* ticket = reinterpret_cast<unsigned int*>(base + kScratchBytes);
    if (cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s) != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(DBQ_ECUDA, "clearing the ticket failed");
    }
    dbq::ScanPackedArgs a;
    a.planes = reinterpret_cast<const uint4*>(planes);
    a.ecount = sizes;
    a.patient = reinterpret_cast<const uint4*>(patient_planes);
    a.pcount = patient_sizes;
    a.n = n;
    a.wp4 = (int)(stride_words / 4);
    dbq::scan_packed_chunking(a.wp4, &a.chunk4, &a.nchunks);
    a.k = k;
    a.cand = reinterpret_cast<dbq::Cand*>(base);
    a.ticket = ticket;
    a.hits = reinterpret_cast<dbq::Hit*>(hits);
    a.counts_out = nullptr;
    a.sup_list = nullptr;
    a.sup_len = nullptr;
    a.group_lists = nullptr;
    a.tickets = nullptr;
    a.counts_in = nullptr;
    const cudaError_t err = dbq::launch_scan_packed(a, grid, s);
    if (err != cudaSuccess) return noalloc_fail(DBQ_ECUDA, cudaGetErrorString(err));
    return DBQ_OK;
}
