// api.cu -- the C ABI of libdbq (declared and documented in include/dbq.h).
//
// Host side only: argument checks, device memory of the database and the
// query workspace, staging of host inputs, and the launches of the kernels
// in pack.cu and scan_packed.cu (and, for half-precision storage,
// scan_f16.cu).  Every step of a query runs in those kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "dbq.h"
#include "kernels.h"
#include "rd.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t err, const char* what)
{
    return fail(DBQ_ECUDA, "%s: %s", what, cudaGetErrorString(err));
}

#define DBQ_CUDA(call)                                               \
    do {                                                             \
        cudaError_t err_ = (call);                                   \
        if (err_ != cudaSuccess) return cuda_fail(err_, #call);      \
    } while (0)

// Keeps the caller's current device unchanged across a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The device address of page-locked host memory (readable by kernels over the
// host link), if p points into such memory and is 16-byte aligned (the
// packing kernels read 16 bytes at a time); else NULL.
const void* pinned_device_view(const void* p)
{
    if (!p || reinterpret_cast<uintptr_t>(p) % 16 != 0) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    if (reinterpret_cast<uintptr_t>(at.devicePointer) % 16 != 0) return nullptr;
    return at.devicePointer;
}

bool threshold_ok(float t) { return std::isfinite(t) && t > 0.0f && t <= 1.0f; }

constexpr int kMaxK = 1024;
constexpr size_t kStageBytes = size_t(256) << 20;   // host-input staging chunk

}  // namespace

int dbq::record_error(int code, const char* msg) { return fail(code, "%s", msg); }

struct dbq_db {
    std::mutex mu;
    int device = 0;
    int nx = 0, ny = 0, nz = 0;
    int64_t v = 0, words = 0, wp = 0;
    int wp4 = 0;
    int64_t n = 0;
    int storage = DBQ_STORE_BITS;
    float t1 = 0.f, t2 = 0.f;
    int n_params = 0;
    uint32_t flags = 0;
    // database
    uint32_t* planes = nullptr;     // [n][2][wp]
    uint32_t* ecount = nullptr;     // [n][2]
    uint16_t* vols16 = nullptr;     // [n][vp] (F16 storage, rows padded with zeros)
    int64_t vp = 0;                 // F16 row length: V rounded up to 1024
    int blocks = 0;                 // F16: 1024-voxel blocks per row
    std::vector<double> params;     // [n][n_params]
    std::vector<uint8_t> loaded;
    int64_t n_loaded = 0;
    bool built = false;
    // query workspace
    void* stage = nullptr;          // device staging for host inputs
    size_t stage_bytes = 0;
    uint32_t* pplanes = nullptr;    // [2][wp] patient planes
    uint32_t* pcount = nullptr;     // [4] patient sizes (2 used)
    dbq::Cand* cand = nullptr;      // [grid][kMaxK]
    dbq::Cand* group_lists = nullptr;   // [ceil(grid/8)][kMaxK] two-level merge
    unsigned int* tickets = nullptr;    // [64] two-level merge counters
    unsigned int* ticket = nullptr;
    dbq::Hit* hits_dev = nullptr;   // [kMaxK]
    dbq::Hit* hits_host = nullptr;  // pinned [kMaxK]
    uint32_t* counts_dev = nullptr; // [n][4], allocated on first db_scan_counts
    // prefilter embeddings (DBQ_FLAG_EMBED)
    int dims = 0;                   // per segmentation
    uint16_t* emb_bf16 = nullptr;   // [n][2][dims]
    uint8_t* emb_f8 = nullptr;      // [n][2][dims]
    float* emb_scale = nullptr;     // [n][2]
    float* emb_nb = nullptr;        // [n][2] squared norms, bf16 rows
    float* emb_nf = nullptr;        // [n][2] squared norms, fp8 rows
    bool sketch = false;            // DBQ_FLAG_SKETCH: count sketches instead of block means
    uint32_t* codes = nullptr;      // [n][2][dims/32] sign codes (DBQ_FLAG_SKETCH)
    uint8_t* codes8 = nullptr;      // [n][2][dims] the same codes as E4M3 0/1 bytes
    float* code_norm = nullptr;     // [n][2] their popcounts
    uint16_t* sk_table = nullptr;   // [V] sketch bucket | sign << 15 of every voxel
    // batch workspace (allocated on first use)
    int bq = 0;                     // capacity in queries
    int bk = 0;                     // capacity in hits per query
    void* bstage = nullptr;         // host patients staged [bq][max bytes]
    size_t bstage_each = 0;
    const void** bptrs = nullptr;   // device [bq] patient pointers
    uint32_t* bplanes = nullptr;    // [bq][2][wp]
    uint32_t* bpcount = nullptr;    // [bq][2]
    uint16_t* bq_bf16 = nullptr;    // [bq][2][dims]
    uint8_t* bq_f8 = nullptr;
    float* bq_scale = nullptr;
    float* bq_nb = nullptr;
    float* bq_nf = nullptr;
    uint32_t* bq_codes = nullptr;   // [bq][2][dims/32]
    uint8_t* bq_codes8 = nullptr;   // [bq][2][dims]
    float* bq_code_norm = nullptr;  // [bq][2]
    float* bdist = nullptr;         // [bq][n]
    int32_t* bcand = nullptr;       // [bq][1024]
    dbq::Cand* brr = nullptr;       // [bq][slices][bk]
    dbq::RerankDedupeWork rrd = {}; // deduplicated re-rank (partial grows with the pairs)
    int rerank_mode = 0;            // DBQ_OPT_RERANK: 0 automatic, 1 per query, 2 deduplicated
    unsigned int* btickets = nullptr;
    dbq::Hit* bhits = nullptr;      // [bq][bk] device
    dbq::Hit* bhits_host = nullptr; // pinned
    int* bstatus = nullptr;         // device status of the tensor-core kernel
    cudaEvent_t ev[6] = {};         // stage boundaries of the last embedding batch
    bool ev_valid = false;
    // nearest-neighbour downsampled copy of another database (0 = none)
    int ds_factor = 0;
    int ds_nx = 0, ds_ny = 0, ds_nz = 0;   // source grid: patients come at this size
    int64_t ds_v = 0, ds_words = 0, ds_wp = 0;
    uint32_t* ds_pplanes = nullptr;        // [2][ds_wp] source-resolution patient planes
    bool sparse = false;            // DBQ_OPT_SPARSE 1 or 2
    int sparse_mode = 0;            // DBQ_OPT_SPARSE: 0, 1, 2 (word-major copy)
    uint4* planes_t = nullptr;      // [2 wp4][n] word-major copy of planes (mode 2)
    bool planes_t_valid = false;    // the copy matches planes
    uint32_t* tcounts = nullptr;    // [n][2] counts of the word-major sparse scan
    uint32_t* plist = nullptr;      // [2][wp4] patient support lists
    uint32_t* plen = nullptr;       // [2]
    uint32_t* bsup = nullptr;       // [bq][2][wp4]
    uint32_t* bsuplen = nullptr;    // [bq][2]
    bool prepared = false;          // a patient sits in pplanes/pcount
    float prep_t1 = 0.f, prep_t2 = 0.f;
    int grid = 1;
    int chunk4 = 1, nchunks = 1;
    size_t bytes_held = 0;

    ~dbq_db()
    {
        cudaFree(planes);
        cudaFree(ecount);
        cudaFree(vols16);
        cudaFree(stage);
        cudaFree(pplanes);
        cudaFree(pcount);
        cudaFree(cand);
        cudaFree(group_lists);
        cudaFree(tickets);
        cudaFree(ticket);
        cudaFree(hits_dev);
        cudaFreeHost(hits_host);
        cudaFree(counts_dev);
        cudaFree(emb_bf16);
        cudaFree(emb_f8);
        cudaFree(emb_scale);
        cudaFree(emb_nb);
        cudaFree(emb_nf);
        cudaFree(codes);
        cudaFree(codes8);
        cudaFree(code_norm);
        cudaFree(sk_table);
        cudaFree(bq_codes);
        cudaFree(bq_codes8);
        cudaFree(bq_code_norm);
        cudaFree(bstage);
        cudaFree(bptrs);
        cudaFree(bplanes);
        cudaFree(bpcount);
        cudaFree(bq_bf16);
        cudaFree(bq_f8);
        cudaFree(bq_scale);
        cudaFree(bq_nb);
        cudaFree(bq_nf);
        cudaFree(bdist);
        cudaFree(bcand);
        cudaFree(brr);
        cudaFree(rrd.hist);
        cudaFree(rrd.tiles);
        cudaFree(rrd.start);
        cudaFree(rrd.uniq);
        cudaFree(rrd.ubeg);
        cudaFree(rrd.nuniq);
        cudaFree(rrd.qof);
        cudaFree(rrd.posof);
        cudaFree(rrd.partial);
        cudaFree(rrd.cnt);
        cudaFree(btickets);
        cudaFree(bhits);
        cudaFreeHost(bhits_host);
        cudaFree(bstatus);
        cudaFree(plist);
        cudaFree(plen);
        cudaFree(planes_t);
        cudaFree(tcounts);
        cudaFree(ds_pplanes);
        cudaFree(bsup);
        cudaFree(bsuplen);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

template <typename T>
int dev_alloc(dbq_db* db, T** p, size_t bytes, const char* what)
{
    cudaError_t err = cudaMalloc(reinterpret_cast<void**>(p), bytes ? bytes : 16);
    if (err != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(DBQ_ENOMEM, "cudaMalloc of %zu bytes for %s failed: %s", bytes, what,
                    cudaGetErrorString(err));
    }
    db->bytes_held += bytes;
    return DBQ_OK;
}

int ensure_stage(dbq_db* db, size_t bytes)
{
    if (db->stage_bytes >= bytes) return DBQ_OK;
    cudaFree(db->stage);
    db->bytes_held -= db->stage_bytes;
    db->stage = nullptr;
    db->stage_bytes = 0;
    int rc = dev_alloc(db, &db->stage, bytes, "input staging");
    if (rc == DBQ_OK) db->stage_bytes = bytes;
    return rc;
}

// Bring a patient into db->pplanes / db->pcount (device), thresholding a
// volume at (t1, t2) or importing caller bit planes.
int prepare_patient(dbq_db* db, const void* patient, int kind, float t1, float t2,
                    cudaStream_t s)
{
    const bool on_dev = is_device_ptr(patient);
    const bool ds = db->ds_factor > 0;
    const int64_t pv = ds ? db->ds_v : db->v;            // patient grid
    const int64_t pwords = ds ? db->ds_words : db->words;
    const int64_t pwp = ds ? db->ds_wp : db->wp;
    uint32_t* pplanes = ds ? db->ds_pplanes : db->pplanes;
    size_t bytes;
    if (kind == DBQ_BITS)
        bytes = (size_t)2 * pwords * sizeof(uint32_t);
    else if (kind == DBQ_F32)
        bytes = (size_t)pv * sizeof(float);
    else if (kind == DBQ_F16)
        bytes = (size_t)pv * sizeof(uint16_t);
    else
        return fail(DBQ_EINVAL, "unknown patient kind %d", kind);
    const void* src = patient;
    const void* view = on_dev ? nullptr : pinned_device_view(patient);
    if (view) {
        src = view;     // page-locked host memory: the packing kernel reads it in place
    } else if (!on_dev) {
        int rc = ensure_stage(db, bytes);
        if (rc) return rc;
        DBQ_CUDA(cudaMemcpyAsync(db->stage, patient, bytes, cudaMemcpyHostToDevice, s));
        src = db->stage;
    }
    DBQ_CUDA(cudaMemsetAsync(db->pcount, 0, 4 * sizeof(uint32_t), s));
    cudaError_t err;
    if (kind == DBQ_BITS)
        err = dbq::launch_import_bits(static_cast<const uint32_t*>(src), pwords, pv, pwp,
                                      pplanes, db->pcount, s);
    else
        err = dbq::launch_pack(src, kind == DBQ_F16, 1, pv, pwp, t1, t2, pplanes, db->pcount, s);
    if (err != cudaSuccess) return cuda_fail(err, "patient packing");
    if (ds) {   // the coarse patient, sampled like the database
        DBQ_CUDA(cudaMemsetAsync(db->pcount, 0, 4 * sizeof(uint32_t), s));
        err = dbq::launch_downsample(db->ds_pplanes, 2, db->ds_wp, db->ds_nx, db->ds_ny,
                                     db->ds_nz, db->ds_factor, db->wp, db->pplanes, db->pcount,
                                     s);
        if (err != cudaSuccess) return cuda_fail(err, "patient downsampling");
    }
    if (db->sparse && db->storage == DBQ_STORE_BITS) {
        err = dbq::launch_support(db->pplanes, 1, db->wp4, db->plist, db->plen, s);
        if (err != cudaSuccess) return cuda_fail(err, "support list launch");
    }
    db->prepared = true;
    db->prep_t1 = t1;
    db->prep_t2 = t2;
    return DBQ_OK;
}

int check_query_args(dbq_db* db, int kind, float* t1, float* t2, int k)
{
    if (!db->built) return fail(DBQ_ESTATE, "database not built (call db_build_masks)");
    if (kind != DBQ_F32 && kind != DBQ_F16 && kind != DBQ_BITS)
        return fail(DBQ_EINVAL, "unknown patient kind %d", kind);
    if (db->storage == DBQ_STORE_BITS) {
        if (std::isnan(*t1)) *t1 = db->t1;
        if (std::isnan(*t2)) *t2 = db->t2;
        if (*t1 != db->t1 || *t2 != db->t2)
            return fail(DBQ_EINVAL,
                        "thresholds (%g, %g) differ from the build thresholds (%g, %g) of a "
                        "bit-packed database",
                        (double)*t1, (double)*t2, (double)db->t1, (double)db->t2);
    } else {
        if (!threshold_ok(*t1) || !threshold_ok(*t2))
            return fail(DBQ_EINVAL, "thresholds must be finite and in (0, 1]");
    }
    if (k < 1) return fail(DBQ_ERANGE, "k = %d must be >= 1", k);
    if (k > db->n || k > kMaxK)
        return fail(DBQ_ERANGE, "k = %d outside [1, min(N=%lld, %d)]", k, (long long)db->n,
                    kMaxK);
    return DBQ_OK;
}

int launch_query(dbq_db* db, int k, dbq::Hit* hits, uint32_t* counts_out, cudaStream_t s)
{
    if (db->storage == DBQ_STORE_BITS) {
        const bool word_major = db->sparse_mode == 2;
        if (word_major) {           // counts over the word-major copy, ranked below
            const int w4 = 2 * (int)db->wp4;
            if (!db->planes_t_valid) {
                cudaError_t err = dbq::launch_transpose_planes(
                    reinterpret_cast<const uint4*>(db->planes), db->n, w4, db->planes_t, s);
                if (err != cudaSuccess) return cuda_fail(err, "word-major copy launch");
                db->planes_t_valid = true;
            }
            DBQ_CUDA(cudaMemsetAsync(db->tcounts, 0, (size_t)db->n * 2 * sizeof(uint32_t), s));
            cudaError_t err = dbq::launch_sparse_t_count(
                db->planes_t, db->n, 1, reinterpret_cast<const uint4*>(db->pplanes),
                (int)db->wp4, db->plist, db->plen, db->tcounts, 0, 2, 1, db->grid, s);
            if (err != cudaSuccess) return cuda_fail(err, "word-major sparse count launch");
        }
        dbq::ScanPackedArgs a;
        a.planes = reinterpret_cast<const uint4*>(db->planes);
        a.ecount = db->ecount;
        a.patient = reinterpret_cast<const uint4*>(db->pplanes);
        a.pcount = db->pcount;
        a.n = db->n;
        a.wp4 = db->wp4;
        a.chunk4 = db->chunk4;
        a.nchunks = db->nchunks;
        a.k = k;
        a.cand = db->cand;
        a.ticket = db->ticket;
        a.hits = hits;
        a.counts_out = counts_out;
        a.sup_list = db->sparse && !word_major ? db->plist : nullptr;
        a.sup_len = db->sparse && !word_major ? db->plen : nullptr;
        a.group_lists = db->grid <= 8 * 63 ? db->group_lists : nullptr;
        a.tickets = db->tickets;
        a.counts_in = word_major ? db->tcounts : nullptr;
        cudaError_t err = dbq::launch_scan_packed(a, db->grid, s);
        if (err != cudaSuccess) return cuda_fail(err, "scan_packed launch");
        return DBQ_OK;
    }
    dbq::ScanF16Args a;
    a.vols = reinterpret_cast<const uint4*>(db->vols16);
    a.patient = db->pplanes;
    a.pcount = db->pcount;
    a.n = db->n;
    a.blocks = db->blocks;
    a.wp = (int)db->wp;
    dbq::scan_f16_chunking(db->blocks, &a.chunk_blocks, &a.nchunks);
    a.k = k;
    const uint32_t th1 = dbq::f16_threshold_bits(db->prep_t1);
    const uint32_t th2 = dbq::f16_threshold_bits(db->prep_t2);
    a.th1x2 = th1 | (th1 << 16);
    a.th2x2 = th2 | (th2 << 16);
    a.cand = db->cand;
    a.ticket = db->ticket;
    a.hits = hits;
    a.counts_out = counts_out;
    cudaError_t err = dbq::launch_scan_f16(a, db->grid, s);
    if (err != cudaSuccess) return cuda_fail(err, "scan_f16 launch");
    return DBQ_OK;
}

}  // namespace

namespace {

constexpr int kBatchQ = 256;      // queries per prefilter group (tensor-core N)
constexpr int kRerankSlices = 4;
constexpr int kRerankDedupeMinQ = 32;    // automatic deduplicated re-rank from this batch size

size_t patient_bytes(const dbq_db* db, int kind)
{
    if (kind == DBQ_BITS) return (size_t)2 * db->words * sizeof(uint32_t);
    if (kind == DBQ_F16) return (size_t)db->v * 2;
    return (size_t)db->v * 4;
}

template <typename T>
int grow(dbq_db* db, T** p, size_t bytes, const char* what)
{
    cudaFree(*p);
    *p = nullptr;
    return dev_alloc(db, p, bytes, what);
}

// Batch workspace for up to kBatchQ queries and k hits each.
int ensure_batch(dbq_db* db, int k)
{
    int rc = DBQ_OK;
    if (db->bq < kBatchQ) {
        const size_t q = kBatchQ;
        rc = grow(db, &db->bptrs, q * sizeof(void*), "batch pointers");
        if (!rc) rc = grow(db, &db->bplanes, q * 2 * db->wp * 4, "batch patient planes");
        if (!rc) rc = grow(db, &db->bpcount, q * 2 * 4, "batch patient sizes");
        if (!rc) rc = grow(db, &db->bhits, q * kMaxK * sizeof(dbq::Hit), "batch hits");
        // one ticket per query, then the sparse re-rank's item counter
        if (!rc) rc = grow(db, &db->btickets, (q + 1) * sizeof(unsigned int), "batch tickets");
        if (!rc) rc = grow(db, &db->bstatus, 16, "status");
        if (!rc) rc = grow(db, &db->bsup, q * 2 * db->wp4 * 4, "batch support lists");
        if (!rc) rc = grow(db, &db->bsuplen, q * 2 * 4, "batch support lengths");
        if (!rc && db->dims) {
            const size_t rows = q * 2;
            rc = grow(db, &db->bq_bf16, rows * db->dims * 2, "query bf16 embeddings");
            if (!rc) rc = grow(db, &db->bq_f8, rows * db->dims, "query fp8 embeddings");
            if (!rc) rc = grow(db, &db->bq_scale, rows * 4, "query scales");
            if (!rc) rc = grow(db, &db->bq_nb, rows * 4, "query bf16 norms");
            if (!rc) rc = grow(db, &db->bq_nf, rows * 4, "query fp8 norms");
            if (!rc && db->sketch)
                rc = grow(db, &db->bq_codes, rows * (db->dims / 32) * 4, "query sign codes");
            if (!rc && db->sketch)
                rc = grow(db, &db->bq_codes8, rows * db->dims, "query code bytes");
            if (!rc && db->sketch)
                rc = grow(db, &db->bq_code_norm, rows * 4, "query code popcounts");
            if (!rc) rc = grow(db, &db->bdist, q * (size_t)db->n * 4, "prefilter distances");
            if (!rc) rc = grow(db, &db->bcand, q * 1024 * 4, "prefilter candidates");
            if (!rc) rc = grow(db, &db->brr, q * kRerankSlices * kMaxK * sizeof(dbq::Cand),
                               "re-rank lists");
            const size_t n = (size_t)db->n, pairs = q * 1024;
            dbq::RerankDedupeWork& w = db->rrd;
            if (!rc) rc = grow(db, &w.hist, n * 4, "re-rank histogram");
            if (!rc) rc = grow(db, &w.tiles, (size_t)dbq::rerank_dedupe_tiles(db->n) * sizeof(uint2),
                               "re-rank tile sums");
            if (!rc) rc = grow(db, &w.start, (n + 1) * 4, "re-rank entry starts");
            if (!rc) rc = grow(db, &w.uniq, n * 4, "re-rank distinct entries");
            if (!rc) rc = grow(db, &w.ubeg, (n + 1) * 4, "re-rank distinct starts");
            if (!rc) rc = grow(db, &w.nuniq, 4, "re-rank distinct count");
            if (!rc) rc = grow(db, &w.qof, pairs * 2, "re-rank pair queries");
            if (!rc) rc = grow(db, &w.posof, pairs * 4, "re-rank pair positions");
            if (!rc) rc = grow(db, &w.cnt, 2 * pairs * 4, "re-rank pair counts");
        }
        if (!rc && !db->bhits_host) {
            cudaError_t err = cudaMallocHost(reinterpret_cast<void**>(&db->bhits_host),
                                             q * kMaxK * sizeof(dbq::Hit));
            if (err != cudaSuccess) {
                cudaGetLastError();
                db->bhits_host = nullptr;
                rc = fail(DBQ_ENOMEM, "pinned host allocation failed");
            }
        }
        if (!rc) {
            cudaError_t err = cudaMemset(db->btickets, 0, (q + 1) * sizeof(unsigned int));
            if (err == cudaSuccess) err = cudaMemset(db->bstatus, 0, 16);
            if (err == cudaSuccess && db->rrd.hist)
                err = cudaMemset(db->rrd.hist, 0, (size_t)db->n * 4);
            if (err == cudaSuccess) err = cudaDeviceSynchronize();
            if (err != cudaSuccess) rc = cuda_fail(err, "batch workspace initialisation");
        }
        if (rc) return rc;
        db->bq = kBatchQ;
    }
    (void)k;
    return DBQ_OK;
}

// Work items per query of the per-query re-rank: every item of a dense
// batch costs the same, so the launch takes ceil(nq x slices / grid) rounds
// of items of c / slices candidates; the count of slices (at least
// kRerankSlices, items of at least 4 candidates, lists [nq][slices][k]
// within the scratch of kBatchQ x kRerankSlices lists) that minimises
// rounds / slices, the smallest of those within 2 %.
int rerank_slices(int nq, int c, int grid)
{
    const int cap = std::max(kRerankSlices, std::min(c / 4, kBatchQ * kRerankSlices / nq));
    int best = kRerankSlices;
    double best_cost = 1e300;
    for (int s = kRerankSlices; s <= cap; ++s) {
        const double cost = (double)(((int64_t)nq * s + grid - 1) / grid) / s;
        if (cost < 0.98 * best_cost) {
            best_cost = cost;
            best = s;
        }
    }
    return std::min(best, c);
}

// Slice counts of the deduplicated re-rank for npairs pairs.
int ensure_rerank_partial(dbq_db* db, int64_t npairs)
{
    const int64_t need =
        (int64_t)2 * dbq::rerank_dedupe_slices((int)db->wp4) * dbq::rerank_dedupe_pstride(npairs);
    if (db->rrd.partial_elems >= need) return DBQ_OK;
    if (db->rrd.partial) db->bytes_held -= (size_t)db->rrd.partial_elems * 2;
    db->rrd.partial_elems = 0;
    int rc = grow(db, &db->rrd.partial, (size_t)need * 2, "re-rank slice counts");
    if (!rc) db->rrd.partial_elems = need;
    return rc;
}

// Threshold (or import) nq patients into bplanes / bpcount.
int prepare_batch(dbq_db* db, int nq, const void* const* patients, int kind, float t1, float t2,
                  cudaStream_t s)
{
    const size_t bytes = patient_bytes(db, kind);
    std::vector<const void*> ptrs((size_t)nq);
    bool any_host = false;
    for (int q = 0; q < nq; ++q) {
        if (!patients[q]) return fail(DBQ_EINVAL, "patient %d is NULL", q);
        any_host |= !is_device_ptr(patients[q]);
    }
    if (any_host && db->bstage_each < bytes) {
        int rc = grow(db, reinterpret_cast<char**>(&db->bstage), (size_t)kBatchQ * bytes,
                      "batch patient staging");
        if (rc) {
            db->bstage_each = 0;
            return rc;
        }
        db->bstage_each = bytes;
    }
    for (int q = 0; q < nq; ++q) {
        if (is_device_ptr(patients[q])) {
            ptrs[q] = patients[q];
        } else {
            char* dst = static_cast<char*>(db->bstage) + (size_t)q * db->bstage_each;
            DBQ_CUDA(cudaMemcpyAsync(dst, patients[q], bytes, cudaMemcpyHostToDevice, s));
            ptrs[q] = dst;
        }
    }
    DBQ_CUDA(cudaMemsetAsync(db->bpcount, 0, (size_t)nq * 2 * 4, s));
    if (kind == DBQ_BITS) {
        for (int q = 0; q < nq; ++q) {
            cudaError_t err = dbq::launch_import_bits(
                static_cast<const uint32_t*>(ptrs[q]), db->words, db->v, db->wp,
                db->bplanes + (size_t)q * 2 * db->wp, db->bpcount + 2 * q, s);
            if (err != cudaSuccess) return cuda_fail(err, "patient import");
        }
    } else {
        DBQ_CUDA(cudaMemcpyAsync(db->bptrs, ptrs.data(), (size_t)nq * sizeof(void*),
                                 cudaMemcpyHostToDevice, s));
        cudaError_t err = dbq::launch_pack_ptrs(db->bptrs, kind == DBQ_F16, nq, db->v, db->wp, t1,
                                                t2, db->bplanes, db->bpcount, s);
        if (err != cudaSuccess) return cuda_fail(err, "batch patient packing");
    }
    if (db->sparse && db->storage == DBQ_STORE_BITS) {
        cudaError_t err = dbq::launch_support(db->bplanes, nq, db->wp4, db->bsup, db->bsuplen, s);
        if (err != cudaSuccess) return cuda_fail(err, "support list launch");
    }
    // the pointer array is pageable: the copy above has been staged already
    return DBQ_OK;
}

// Prefilter for the nq prepared patients: embeddings, tensor-core distances,
// candidate selection into bdist / bcand.
void mark(dbq_db* db, int i, cudaStream_t s)
{
    if (!db->ev[0]) {
        for (cudaEvent_t& e : db->ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                e = nullptr;
            }
    }
    if (db->ev[i]) cudaEventRecord(db->ev[i], s);
}

int run_prefilter(dbq_db* db, int nq, int mode, int c, cudaStream_t s)
{
    mark(db, 1, s);
    cudaError_t err =
        db->sketch
            ? dbq::launch_sketch(db->bplanes, nq, db->wp, db->words, db->sk_table, db->bq_bf16,
                                 db->bq_f8,
                                 db->bq_scale, db->bq_nb, db->bq_nf, db->bq_codes, db->bq_codes8,
                                 db->bq_code_norm, s)
            : dbq::launch_embed(db->bplanes, nq, db->wp, db->nx, db->ny, db->nz, db->bq_bf16,
                                db->bq_f8, db->bq_scale, db->bq_nb, db->bq_nf, s);
    if (err != cudaSuccess) return cuda_fail(err, "query embedding launch");
    mark(db, 2, s);
    {
        const bool ham = mode == DBQ_MODE_HASH;
        const int fp8 = mode == DBQ_MODE_EMBED_FP8;
        dbq::GemmArgs g;
        g.e_bf16 = db->emb_bf16;
        g.e_f8 = ham ? db->codes8 : db->emb_f8;
        g.enorm = ham ? db->code_norm : (fp8 ? db->emb_nf : db->emb_nb);
        g.escale = db->emb_scale;
        g.q_bf16 = db->bq_bf16;
        g.q_f8 = ham ? db->bq_codes8 : db->bq_f8;
        g.qnorm = ham ? db->bq_code_norm : (fp8 ? db->bq_nf : db->bq_nb);
        g.qscale = db->bq_scale;
        g.n = db->n;
        g.nq = nq;
        g.dims = db->dims;
        g.dist = db->bdist;
        g.status = db->bstatus;
        const int kind = ham ? dbq::kGemmHamming : (fp8 ? dbq::kGemmFp8 : dbq::kGemmBf16);
        err = dbq::launch_prefilter_gemm(g, kind, db->grid, s);
        if (err != cudaSuccess) return cuda_fail(err, "prefilter GEMM launch");
    }
    mark(db, 3, s);
    if (c > 0) {
        err = dbq::launch_select_smallest(db->bdist, nq, db->n, c, db->bcand, s);
        if (err != cudaSuccess) return cuda_fail(err, "candidate selection launch");
    }
    mark(db, 4, s);
    return DBQ_OK;
}

int check_status(dbq_db* db, cudaStream_t s)
{
    int st[4] = {0, 0, 0, 0};
    DBQ_CUDA(cudaMemcpyAsync(st, db->bstatus, sizeof st, cudaMemcpyDeviceToHost, s));
    DBQ_CUDA(cudaStreamSynchronize(s));
    if (st[0] != 0) {
        cudaMemsetAsync(db->bstatus, 0, 16, s);
        cudaStreamSynchronize(s);
        return fail(DBQ_ETIMEOUT, "tensor-core prefilter gave up waiting (role %d)", st[0]);
    }
    return DBQ_OK;
}

int check_prefilter_args(dbq_db* db, int mode, int c, int k)
{
    if (!db->built) return fail(DBQ_ESTATE, "database not built (call db_build_masks)");
    if (!db->dims)
        return fail(DBQ_ESTATE, "database has no embeddings (DBQ_FLAG_EMBED or DBQ_FLAG_SKETCH)");
    if (mode != DBQ_MODE_EMBED_BF16 && mode != DBQ_MODE_EMBED_FP8 && mode != DBQ_MODE_HASH)
        return fail(DBQ_EINVAL, "unknown prefilter mode %d", mode);
    if (mode == DBQ_MODE_HASH && !db->sketch)
        return fail(DBQ_ESTATE, "hash codes need a database built with DBQ_FLAG_SKETCH");
    if (mode == DBQ_MODE_EMBED_FP8 && db->dims % 128)
        return fail(DBQ_EINVAL, "FP8 prefilter needs a multiple of 128 embedding dims");
    if (mode == DBQ_MODE_EMBED_BF16 && db->dims % 64)
        return fail(DBQ_EINVAL, "bf16 prefilter needs a multiple of 64 embedding dims");
    if (c < 1 || c > 1024 || c > db->n || c < k)
        return fail(DBQ_ERANGE, "n_candidates %d outside [k, min(N, 1024)]", c);
    return DBQ_OK;
}

}  // namespace

struct dbq_plan {
    std::vector<dbq_db*> dbs;
    int device = 0;
    int maxq = 0, k = 0;
    int items_per_sm = 4;
    int sms = 1;
    int64_t max_wp = 0;
    int max_slices = 64;
    uint32_t* planes = nullptr;       // [maxq][2][max_wp]
    uint32_t* pcount = nullptr;       // [maxq][2]
    uint32_t* sup = nullptr;          // [maxq][2][max_wp / 4]
    uint32_t* suplen = nullptr;       // [maxq][2]
    dbq::Cand* scratch = nullptr;     // [maxq][max_slices][k]
    unsigned int* tickets = nullptr;  // [maxq]
    unsigned int* counter = nullptr;
    dbq::QueryTask* tasks_dev = nullptr;
    dbq::QueryTask* tasks_host = nullptr;   // pinned
    int2* items_dev = nullptr;
    int2* items_host = nullptr;             // pinned
    const void** ptrs_dev = nullptr;
    const void** ptrs_host = nullptr;       // pinned
    cudaEvent_t copied = nullptr;
    bool copy_pending = false;
    // tensor-core path for databases queried by many dense queries at once
    int tc_min = 16;                  // queries per database that switch it on (0 = never)
    std::vector<int> tc_min_db;       // per-database override, -1 = tc_min
    int tc_rows = 0;                  // queries per tensor-core launch (0 = unavailable)
    uint32_t* tc_counts = nullptr;    // [2][tc_rows][stride of the largest n] intersections
    unsigned long long tc_stall_ns = 0;   // DBQ_PLAN_TEST_STALL_NS
    int* tc_status = nullptr;         // nonzero after a timed-out wait
    ~dbq_plan()
    {
        cudaFree(tc_counts);
        cudaFree(tc_status);
        cudaFree(planes);
        cudaFree(pcount);
        cudaFree(sup);
        cudaFree(suplen);
        cudaFree(scratch);
        cudaFree(tickets);
        cudaFree(counter);
        cudaFree(tasks_dev);
        cudaFreeHost(tasks_host);
        cudaFree(items_dev);
        cudaFreeHost(items_host);
        cudaFree(ptrs_dev);
        cudaFreeHost(ptrs_host);
        if (copied) cudaEventDestroy(copied);
    }
};

// Forward-model solver (rd.h): the tissue map, its face coefficients and
// the ping-pong fields of one batch of simulations.
struct rd_solver {
    int device = 0;
    int nx = 0, ny = 0, nz = 0;
    int64_t v = 0;
    int batch = 0;
    std::vector<float> tissue;      // host copy (seed checks, max)
    double m_max = 0.0;
    float* m_dev = nullptr;
    float* hx = nullptr;
    float* hy = nullptr;
    float* hz = nullptr;
    float* hym = nullptr;
    unsigned int* tile_any = nullptr;
    dbq::RdSim* sims = nullptr;     // [batch]
    float* buf0 = nullptr;          // [batch][V]
    float* buf1 = nullptr;
    unsigned long long* updates = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double stats[4] = {0, 0, 0, 0};
    bool ran = false;
    std::mutex mu;

    ~rd_solver()
    {
        cudaFree(m_dev);
        cudaFree(hx);
        cudaFree(hy);
        cudaFree(hz);
        cudaFree(hym);
        cudaFree(tile_any);
        cudaFree(sims);
        cudaFree(buf0);
        cudaFree(buf1);
        cudaFree(updates);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

namespace {

template <typename T>
int rd_alloc(T** p, size_t bytes, const char* what)
{
    if (cudaMalloc(reinterpret_cast<void**>(p), bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(DBQ_ENOMEM, "device allocation of %zu bytes for %s failed", bytes, what);
    }
    return DBQ_OK;
}

// Explicit-Euler step count of the scheme in rd.h (binary64, no contraction).
int64_t rd_step_count(double t_end, double dw, double rho, double m_max, double cfl)
{
    if (!(t_end > 0.0)) return 0;
    const double rate = 6.0 * dw * m_max + rho;
    const double n = std::ceil(t_end * rate / cfl);
    return n < 1.0 ? 1 : (int64_t)n;
}

}  // namespace

extern "C" {

const char* db_last_error(void) { return g_last_error.c_str(); }

int db_create(dbq_db** out, int nx, int ny, int nz, int64_t capacity, int storage, float t1,
              float t2, int n_params, uint32_t flags)
{
    if (!out) return fail(DBQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(DBQ_EINVAL, "grid dimensions must be >= 1");
    const int64_t v = (int64_t)nx * ny * nz;
    if (v >= (int64_t(1) << 31)) return fail(DBQ_EINVAL, "volume of %lld voxels too large",
                                             (long long)v);
    if (capacity < 1) return fail(DBQ_EINVAL, "capacity must be >= 1");
    if (storage != DBQ_STORE_BITS && storage != DBQ_STORE_F16)
        return fail(DBQ_EINVAL, "unknown storage %d", storage);
    if (storage == DBQ_STORE_BITS && (!threshold_ok(t1) || !threshold_ok(t2)))
        return fail(DBQ_EINVAL, "build thresholds must be finite and in (0, 1]");
    if (n_params < 0 || n_params > 64) return fail(DBQ_EINVAL, "n_params must be in [0, 64]");
    if (flags & ~(DBQ_FLAG_EMBED | DBQ_FLAG_SKETCH))
        return fail(DBQ_EINVAL, "unknown flags 0x%x", flags);
    if ((flags & DBQ_FLAG_EMBED) && (flags & DBQ_FLAG_SKETCH))
        return fail(DBQ_EINVAL, "DBQ_FLAG_EMBED and DBQ_FLAG_SKETCH exclude each other");
    if ((flags & DBQ_FLAG_SKETCH) && storage != DBQ_STORE_BITS)
        return fail(DBQ_EINVAL, "sketch embeddings need bit-packed storage");
    if ((flags & DBQ_FLAG_EMBED) &&
        (storage != DBQ_STORE_BITS || !dbq::embed_supported(nx, ny, nz)))
        return fail(DBQ_EINVAL,
                    "embeddings need bit-packed storage, nx a multiple of 32 and ny, nz "
                    "multiples of 8");

    int dev = 0;
    DBQ_CUDA(cudaGetDevice(&dev));
    dbq_db* db = new (std::nothrow) dbq_db;
    if (!db) return fail(DBQ_ENOMEM, "host allocation failed");
    db->device = dev;
    db->nx = nx;
    db->ny = ny;
    db->nz = nz;
    db->v = v;
    db->words = (v + 31) / 32;
    if (storage == DBQ_STORE_F16) {
        db->blocks = (int)((v + 1023) / 1024);
        db->vp = (int64_t)db->blocks * 1024;
        db->wp = (int64_t)db->blocks * 32;     // patient planes cover whole blocks
    } else {
        db->wp = (db->words + 3) / 4 * 4;
    }
    db->wp4 = (int)(db->wp / 4);
    db->n = capacity;
    db->storage = storage;
    db->t1 = t1;
    db->t2 = t2;
    db->n_params = n_params;
    db->flags = flags;
    try {
        db->params.assign((size_t)capacity * n_params, 0.0);
        db->loaded.assign((size_t)capacity, 0);
    } catch (...) {
        delete db;
        return fail(DBQ_ENOMEM, "host allocation of per-entry metadata failed");
    }
    int rc = DBQ_OK;
    if (storage == DBQ_STORE_BITS) {
        rc = dev_alloc(db, &db->planes, (size_t)capacity * 2 * db->wp * sizeof(uint32_t),
                       "bit planes");
        if (!rc)
            rc = dev_alloc(db, &db->ecount, (size_t)capacity * 2 * sizeof(uint32_t),
                           "mask sizes");
    } else {
        rc = dev_alloc(db, &db->vols16, (size_t)capacity * db->vp * sizeof(uint16_t),
                       "binary16 volumes");
    }
    if (!rc && (flags & (DBQ_FLAG_EMBED | DBQ_FLAG_SKETCH))) {
        db->sketch = (flags & DBQ_FLAG_SKETCH) != 0;
        db->dims = db->sketch ? dbq::sketch_dims() : dbq::embed_dims(nx, ny, nz);
        const size_t rows = (size_t)capacity * 2;
        rc = dev_alloc(db, &db->emb_bf16, rows * db->dims * 2, "bf16 embeddings");
        if (!rc) rc = dev_alloc(db, &db->emb_f8, rows * db->dims, "fp8 embeddings");
        if (!rc) rc = dev_alloc(db, &db->emb_scale, rows * 4, "fp8 scales");
        if (!rc) rc = dev_alloc(db, &db->emb_nb, rows * 4, "bf16 norms");
        if (!rc) rc = dev_alloc(db, &db->emb_nf, rows * 4, "fp8 norms");
        if (!rc && db->sketch)
            rc = dev_alloc(db, &db->codes, rows * (db->dims / 32) * 4, "sign codes");
        if (!rc && db->sketch) rc = dev_alloc(db, &db->codes8, rows * db->dims, "code bytes");
        if (!rc && db->sketch) rc = dev_alloc(db, &db->code_norm, rows * 4, "code popcounts");
        if (!rc && db->sketch) rc = dev_alloc(db, &db->sk_table, (size_t)v * 2, "sketch table");
        if (!rc && db->sketch) {
            cudaError_t err = dbq::launch_sketch_table(v, db->sk_table, nullptr);
            if (err == cudaSuccess) err = cudaDeviceSynchronize();
            if (err != cudaSuccess) rc = cuda_fail(err, "sketch table");
        }
    }
    db->grid = dbq::scan_packed_grid(dev);
    dbq::scan_packed_chunking(db->wp4, &db->chunk4, &db->nchunks);
    if (!rc) rc = dev_alloc(db, &db->pplanes, (size_t)2 * db->wp * sizeof(uint32_t), "patient");
    if (!rc) rc = dev_alloc(db, &db->pcount, 4 * sizeof(uint32_t), "patient sizes");
    if (!rc) rc = dev_alloc(db, &db->plist, (size_t)2 * db->wp4 * sizeof(uint32_t), "support lists");
    if (!rc) rc = dev_alloc(db, &db->plen, 4 * sizeof(uint32_t), "support lengths");
    if (!rc)
        rc = dev_alloc(db, &db->cand, (size_t)db->grid * kMaxK * sizeof(dbq::Cand),
                       "candidate lists");
    if (!rc) rc = dev_alloc(db, &db->ticket, sizeof(unsigned int), "ticket");
    if (!rc)
        rc = dev_alloc(db, &db->group_lists,
                       (size_t)((db->grid + 7) / 8) * kMaxK * sizeof(dbq::Cand), "group lists");
    if (!rc) rc = dev_alloc(db, &db->tickets, 64 * sizeof(unsigned int), "merge tickets");
    if (!rc) rc = dev_alloc(db, &db->hits_dev, (size_t)kMaxK * sizeof(dbq::Hit), "hits");
    if (!rc) {
        cudaError_t err = cudaMallocHost(reinterpret_cast<void**>(&db->hits_host),
                                         (size_t)kMaxK * sizeof(dbq::Hit));
        if (err != cudaSuccess) {
            cudaGetLastError();
            db->hits_host = nullptr;
            rc = fail(DBQ_ENOMEM, "pinned host allocation failed");
        }
    }
    if (!rc) {
        cudaError_t err = cudaMemset(db->ticket, 0, sizeof(unsigned int));
        if (err == cudaSuccess) err = cudaMemset(db->tickets, 0, 64 * sizeof(unsigned int));
        if (err == cudaSuccess && db->ecount)
            err = cudaMemset(db->ecount, 0, (size_t)capacity * 2 * sizeof(uint32_t));
        if (err == cudaSuccess && db->vols16)   // zero padding never reaches a threshold
            err = cudaMemset(db->vols16, 0, (size_t)capacity * db->vp * sizeof(uint16_t));
        if (err == cudaSuccess) err = cudaDeviceSynchronize();
        if (err != cudaSuccess) rc = cuda_fail(err, "workspace initialisation");
    }
    if (rc) {
        delete db;
        return rc;
    }
    *out = db;
    return DBQ_OK;
}

int db_load_volumes(dbq_db* db, int64_t first, int64_t count, const void* vols, int kind,
                    const double* params, void* stream)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    std::lock_guard<std::mutex> lock(db->mu);
    if (count == 0) return DBQ_OK;
    if (!vols) return fail(DBQ_EINVAL, "vols is NULL");
    if (first < 0 || count < 0 || first + count > db->n)
        return fail(DBQ_ERANGE, "entries [%lld, %lld) outside [0, %lld)", (long long)first,
                    (long long)(first + count), (long long)db->n);
    if (kind != DBQ_F32 && kind != DBQ_F16)
        return fail(DBQ_EINVAL, "volumes must be DBQ_F32 or DBQ_F16");
    DeviceGuard guard(db->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t esz = kind == DBQ_F16 ? 2 : 4;
    const size_t vol_bytes = (size_t)db->v * esz;
    const bool on_dev = is_device_ptr(vols);
    int64_t per_chunk = count;
    if (!on_dev) {
        per_chunk = (int64_t)(kStageBytes / vol_bytes);
        if (per_chunk < 1) per_chunk = 1;
        if (per_chunk > count) per_chunk = count;
        int rc = ensure_stage(db, (size_t)per_chunk * vol_bytes);
        if (rc) return rc;
    }
    db->built = false;
    for (int64_t c0 = 0; c0 < count; c0 += per_chunk) {
        const int64_t cn = (count - c0) < per_chunk ? (count - c0) : per_chunk;
        const char* src = static_cast<const char*>(vols) + (size_t)c0 * vol_bytes;
        if (!on_dev) {
            DBQ_CUDA(cudaMemcpyAsync(db->stage, src, (size_t)cn * vol_bytes,
                                     cudaMemcpyHostToDevice, s));
            src = static_cast<const char*>(db->stage);
        }
        const int64_t e0 = first + c0;
        if (db->storage == DBQ_STORE_BITS) {
            DBQ_CUDA(cudaMemsetAsync(db->ecount + 2 * e0, 0, (size_t)cn * 2 * sizeof(uint32_t),
                                     s));
            cudaError_t err = dbq::launch_pack(src, kind == DBQ_F16, cn, db->v, db->wp, db->t1,
                                               db->t2, db->planes + e0 * 2 * db->wp,
                                               db->ecount + 2 * e0, s);
            if (err != cudaSuccess) return cuda_fail(err, "pack launch");
        } else {
            uint16_t* dst = db->vols16 + e0 * db->vp;
            cudaError_t err = dbq::launch_rows_to_f16(src, kind == DBQ_F16, cn, db->v, db->vp,
                                                      dst, s);
            if (err != cudaSuccess) return cuda_fail(err, "binary16 storage launch");
        }
    }
    if (!on_dev) DBQ_CUDA(cudaStreamSynchronize(s));   // the caller may reuse its buffer
    for (int64_t e = first; e < first + count; ++e) {
        if (!db->loaded[e]) {
            db->loaded[e] = 1;
            ++db->n_loaded;
        }
        if (db->n_params) {
            double* dst = &db->params[(size_t)e * db->n_params];
            if (params)
                std::memcpy(dst, params + (size_t)(e - first) * db->n_params,
                            sizeof(double) * db->n_params);
            else
                std::memset(dst, 0, sizeof(double) * db->n_params);
        }
    }
    return DBQ_OK;
}

int db_build_masks(dbq_db* db, void* stream)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    std::lock_guard<std::mutex> lock(db->mu);
    if (db->n_loaded != db->n)
        return fail(DBQ_ESTATE, "%lld of %lld entries loaded", (long long)db->n_loaded,
                    (long long)db->n);
    DeviceGuard guard(db->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (db->flags & DBQ_FLAG_EMBED) {
        cudaError_t err = dbq::launch_embed(db->planes, db->n, db->wp, db->nx, db->ny, db->nz,
                                            db->emb_bf16, db->emb_f8, db->emb_scale, db->emb_nb,
                                            db->emb_nf, s);
        if (err != cudaSuccess) return cuda_fail(err, "embedding launch");
    } else if (db->flags & DBQ_FLAG_SKETCH) {
        cudaError_t err = dbq::launch_sketch(db->planes, db->n, db->wp, db->words, db->sk_table,
                                             db->emb_bf16,
                                             db->emb_f8, db->emb_scale, db->emb_nb, db->emb_nf,
                                             db->codes, db->codes8, db->code_norm, s);
        if (err != cudaSuccess) return cuda_fail(err, "sketch launch");
    }
    db->planes_t_valid = false;
    if (db->sparse_mode == 2) {     // the word-major copy follows the planes
        cudaError_t err = dbq::launch_transpose_planes(reinterpret_cast<const uint4*>(db->planes),
                                                       db->n, 2 * (int)db->wp4, db->planes_t, s);
        if (err != cudaSuccess) return cuda_fail(err, "word-major copy launch");
        db->planes_t_valid = true;
    }
    DBQ_CUDA(cudaStreamSynchronize(s));
    db->built = true;
    return DBQ_OK;
}

int db_query_async(dbq_db* db, const void* patient_dev, int kind, float t1, float t2, int k,
                   dbq_hit* hits_dev, void* stream)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    if (!patient_dev || !hits_dev) return fail(DBQ_EINVAL, "NULL pointer argument");
    std::lock_guard<std::mutex> lock(db->mu);
    int rc = check_query_args(db, kind, &t1, &t2, k);
    if (rc) return rc;
    DeviceGuard guard(db->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
    if (!is_device_ptr(patient_dev) || !is_device_ptr(hits_dev))
        return fail(DBQ_EINVAL, "db_query_async needs device pointers");
    if (reinterpret_cast<uintptr_t>(hits_dev) % 8)
        return fail(DBQ_EINVAL, "hits_dev must be 8-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    rc = prepare_patient(db, patient_dev, kind, t1, t2, s);
    if (rc) return rc;
    return launch_query(db, k, reinterpret_cast<dbq::Hit*>(hits_dev), nullptr, s);
}

int db_prepare_patient(dbq_db* db, const void* patient_dev, int kind, float t1, float t2,
                       void* stream)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    if (!patient_dev) return fail(DBQ_EINVAL, "NULL pointer argument");
    std::lock_guard<std::mutex> lock(db->mu);
    int rc = check_query_args(db, kind, &t1, &t2, 1);
    if (rc) return rc;
    DeviceGuard guard(db->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
    if (!is_device_ptr(patient_dev))
        return fail(DBQ_EINVAL, "db_prepare_patient needs a device pointer");
    return prepare_patient(db, patient_dev, kind, t1, t2, reinterpret_cast<cudaStream_t>(stream));
}

int db_query_prepared(dbq_db* db, int k, dbq_hit* hits_dev, void* stream)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    if (!hits_dev) return fail(DBQ_EINVAL, "NULL pointer argument");
    std::lock_guard<std::mutex> lock(db->mu);
    if (!db->prepared) return fail(DBQ_ESTATE, "no patient prepared");
    float t1 = db->prep_t1, t2 = db->prep_t2;
    int rc = check_query_args(db, DBQ_BITS, &t1, &t2, k);
    if (rc) return rc;
    DeviceGuard guard(db->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
    if (!is_device_ptr(hits_dev) || reinterpret_cast<uintptr_t>(hits_dev) % 8)
        return fail(DBQ_EINVAL, "hits_dev must be 8-byte aligned device memory");
    return launch_query(db, k, reinterpret_cast<dbq::Hit*>(hits_dev), nullptr,
                        reinterpret_cast<cudaStream_t>(stream));
}

int db_query(dbq_db* db, const void* patient, int kind, float t1, float t2, int k,
             dbq_hit* hits, double* params, void* stream)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    if (!patient || !hits) return fail(DBQ_EINVAL, "NULL pointer argument");
    std::lock_guard<std::mutex> lock(db->mu);
    int rc = check_query_args(db, kind, &t1, &t2, k);
    if (rc) return rc;
    DeviceGuard guard(db->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    rc = prepare_patient(db, patient, kind, t1, t2, s);
    if (rc) return rc;
    rc = launch_query(db, k, db->hits_dev, nullptr, s);
    if (rc) return rc;
    DBQ_CUDA(cudaMemcpyAsync(db->hits_host, db->hits_dev, (size_t)k * sizeof(dbq::Hit),
                             cudaMemcpyDeviceToHost, s));
    DBQ_CUDA(cudaStreamSynchronize(s));
    // every check before the first byte of output is written
    const dbq_hit* got = reinterpret_cast<const dbq_hit*>(db->hits_host);
    for (int j = 0; j < k; ++j)
        if (got[j].index < 0 || got[j].index >= db->n)
            return fail(DBQ_ECUDA, "kernel returned index %lld", (long long)got[j].index);
    std::memcpy(hits, got, (size_t)k * sizeof(dbq_hit));
    if (params && db->n_params)
        for (int j = 0; j < k; ++j)
            std::memcpy(params + (size_t)j * db->n_params,
                        &db->params[(size_t)got[j].index * db->n_params],
                        sizeof(double) * db->n_params);
    return DBQ_OK;
}

int db_scan_counts(dbq_db* db, const void* patient, int kind, float t1, float t2,
                   uint32_t* counts, uint32_t* pcount, void* stream)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    if (!patient || !counts || !pcount) return fail(DBQ_EINVAL, "NULL pointer argument");
    std::lock_guard<std::mutex> lock(db->mu);
    int rc = check_query_args(db, kind, &t1, &t2, 1);
    if (rc) return rc;
    DeviceGuard guard(db->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    rc = prepare_patient(db, patient, kind, t1, t2, s);
    if (rc) return rc;
    const bool dev_out = is_device_ptr(counts) && reinterpret_cast<uintptr_t>(counts) % 16 == 0;
    uint32_t* dst = counts;
    if (!dev_out) {
        if (!db->counts_dev) {
            rc = dev_alloc(db, &db->counts_dev, (size_t)db->n * 4 * sizeof(uint32_t), "counts");
            if (rc) return rc;
        }
        dst = db->counts_dev;
    }
    rc = launch_query(db, 1, nullptr, dst, s);
    if (rc) return rc;
    if (dst != counts)
        DBQ_CUDA(cudaMemcpyAsync(counts, dst, (size_t)db->n * 4 * sizeof(uint32_t),
                                 cudaMemcpyDefault, s));
    DBQ_CUDA(cudaMemcpyAsync(pcount, db->pcount, 2 * sizeof(uint32_t), cudaMemcpyDefault, s));
    DBQ_CUDA(cudaStreamSynchronize(s));
    return DBQ_OK;
}

int db_get_masks(dbq_db* db, int64_t first, int64_t count, uint32_t* planes, uint32_t* sizes,
                 void* stream)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    std::lock_guard<std::mutex> lock(db->mu);
    if (db->storage != DBQ_STORE_BITS) return fail(DBQ_ESTATE, "not a bit-packed database");
    if (first < 0 || count < 0 || first + count > db->n)
        return fail(DBQ_ERANGE, "entries outside [0, N)");
    if (count == 0) return DBQ_OK;
    if (!planes) return fail(DBQ_EINVAL, "planes is NULL");
    DeviceGuard guard(db->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // [count*2] rows of `words` words out of rows of `wp` words
    DBQ_CUDA(cudaMemcpy2DAsync(planes, (size_t)db->words * 4, db->planes + first * 2 * db->wp,
                               (size_t)db->wp * 4, (size_t)db->words * 4, (size_t)count * 2,
                               cudaMemcpyDefault, s));
    if (sizes)
        DBQ_CUDA(cudaMemcpyAsync(sizes, db->ecount + 2 * first, (size_t)count * 2 * 4,
                                 cudaMemcpyDefault, s));
    DBQ_CUDA(cudaStreamSynchronize(s));
    return DBQ_OK;
}

int db_get_embeddings(dbq_db* db, int64_t first, int64_t count, uint16_t* bf16, uint8_t* e4m3,
                      float* scale, float* norm_bf16, float* norm_fp8, void* stream)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    std::lock_guard<std::mutex> lock(db->mu);
    if (!db->dims)
        return fail(DBQ_ESTATE, "database has no embeddings (DBQ_FLAG_EMBED or DBQ_FLAG_SKETCH)");
    if (!db->built) return fail(DBQ_ESTATE, "database not built (call db_build_masks)");
    if (first < 0 || count < 0 || first + count > db->n)
        return fail(DBQ_ERANGE, "entries outside [0, N)");
    if (count == 0) return DBQ_OK;
    DeviceGuard guard(db->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t rows = (size_t)count * 2, r0 = (size_t)first * 2;
    if (bf16)
        DBQ_CUDA(cudaMemcpyAsync(bf16, db->emb_bf16 + r0 * db->dims, rows * db->dims * 2,
                                 cudaMemcpyDefault, s));
    if (e4m3)
        DBQ_CUDA(cudaMemcpyAsync(e4m3, db->emb_f8 + r0 * db->dims, rows * db->dims,
                                 cudaMemcpyDefault, s));
    if (scale)
        DBQ_CUDA(cudaMemcpyAsync(scale, db->emb_scale + r0, rows * 4, cudaMemcpyDefault, s));
    if (norm_bf16)
        DBQ_CUDA(cudaMemcpyAsync(norm_bf16, db->emb_nb + r0, rows * 4, cudaMemcpyDefault, s));
    if (norm_fp8)
        DBQ_CUDA(cudaMemcpyAsync(norm_fp8, db->emb_nf + r0, rows * 4, cudaMemcpyDefault, s));
    DBQ_CUDA(cudaStreamSynchronize(s));
    return DBQ_OK;
}

int db_get_codes(dbq_db* db, int64_t first, int64_t count, uint32_t* codes, void* stream)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    std::lock_guard<std::mutex> lock(db->mu);
    if (!db->sketch) return fail(DBQ_ESTATE, "database has no sign codes (DBQ_FLAG_SKETCH)");
    if (!db->built) return fail(DBQ_ESTATE, "database not built (call db_build_masks)");
    if (first < 0 || count < 0 || first + count > db->n)
        return fail(DBQ_ERANGE, "entries outside [0, N)");
    if (count == 0) return DBQ_OK;
    if (!codes) return fail(DBQ_EINVAL, "codes is NULL");
    DeviceGuard guard(db->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t row_words = (size_t)db->dims / 32;
    DBQ_CUDA(cudaMemcpyAsync(codes, db->codes + (size_t)first * 2 * row_words,
                             (size_t)count * 2 * row_words * 4, cudaMemcpyDefault, s));
    DBQ_CUDA(cudaStreamSynchronize(s));
    return DBQ_OK;
}

int db_create_downsampled(dbq_db** out, dbq_db* src, int factor)
{
    if (!out || !src) return fail(DBQ_EINVAL, "NULL pointer argument");
    *out = nullptr;
    std::lock_guard<std::mutex> lock(src->mu);
    if (src->storage != DBQ_STORE_BITS || !src->built)
        return fail(DBQ_ESTATE, "source must be a built bit-packed database");
    if (src->ds_factor) return fail(DBQ_ESTATE, "source is itself downsampled");
    if (factor < 2 || factor > 16 || src->nx % factor || src->ny % factor || src->nz % factor)
        return fail(DBQ_EINVAL, "factor must be in [2, 16] and divide the grid");
    DeviceGuard guard(src->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", src->device);
    dbq_db* db = nullptr;
    int rc = db_create(&db, src->nx / factor, src->ny / factor, src->nz / factor, src->n,
                       DBQ_STORE_BITS, src->t1, src->t2, src->n_params, 0);
    if (rc) return rc;
    db->ds_factor = factor;
    db->ds_nx = src->nx;
    db->ds_ny = src->ny;
    db->ds_nz = src->nz;
    db->ds_v = src->v;
    db->ds_words = src->words;
    db->ds_wp = src->wp;
    rc = dev_alloc(db, &db->ds_pplanes, (size_t)2 * src->wp * 4, "source-resolution patient");
    if (rc) {
        delete db;
        return rc;
    }
    cudaError_t err = cudaMemset(db->ecount, 0, (size_t)db->n * 2 * 4);
    if (err == cudaSuccess)
        err = dbq::launch_downsample(src->planes, src->n * 2, src->wp, src->nx, src->ny, src->nz,
                                     factor, db->wp, db->planes, db->ecount, nullptr);
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        delete db;
        return cuda_fail(err, "downsampling");
    }
    db->params = src->params;
    std::fill(db->loaded.begin(), db->loaded.end(), 1);
    db->n_loaded = db->n;
    db->built = true;
    *out = db;
    return DBQ_OK;
}

int db_prefilter(dbq_db* db, int nq, const void* const* patients, int kind, int mode,
                 int n_candidates, float* dist, int32_t* cand, void* stream)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    if (!patients) return fail(DBQ_EINVAL, "patients is NULL");
    std::lock_guard<std::mutex> lock(db->mu);
    if (nq < 1 || nq > kBatchQ) return fail(DBQ_ERANGE, "nq must be in [1, %d]", kBatchQ);
    int rc = check_prefilter_args(db, mode, cand ? n_candidates : 1, 1);
    if (rc) return rc;
    if (kind != DBQ_F32 && kind != DBQ_F16 && kind != DBQ_BITS)
        return fail(DBQ_EINVAL, "unknown patient kind %d", kind);
    DeviceGuard guard(db->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    rc = ensure_batch(db, 1);
    if (!rc) rc = prepare_batch(db, nq, patients, kind, db->t1, db->t2, s);
    if (!rc) rc = run_prefilter(db, nq, mode, cand ? n_candidates : 0, s);
    if (rc) return rc;
    if (dist)
        DBQ_CUDA(cudaMemcpyAsync(dist, db->bdist, (size_t)nq * db->n * 4, cudaMemcpyDefault, s));
    if (cand)
        DBQ_CUDA(cudaMemcpyAsync(cand, db->bcand, (size_t)nq * n_candidates * 4,
                                 cudaMemcpyDefault, s));
    return check_status(db, s);
}

int db_query_batch(dbq_db* const* dbs, const int* db_of_query, int nq,
                   const void* const* patients, int kind, const float* t1, const float* t2,
                   int k, int mode, int n_candidates, dbq_hit* hits, double* params,
                   void* stream)
{
    if (!dbs || !db_of_query || !patients || !hits) return fail(DBQ_EINVAL, "NULL argument");
    if (nq < 0) return fail(DBQ_EINVAL, "nq < 0");
    if (mode != DBQ_MODE_EXACT && mode != DBQ_MODE_EMBED_BF16 && mode != DBQ_MODE_EMBED_FP8 &&
        mode != DBQ_MODE_HASH)
        return fail(DBQ_EINVAL, "unknown mode %d", mode);
    if (kind != DBQ_F32 && kind != DBQ_F16 && kind != DBQ_BITS)
        return fail(DBQ_EINVAL, "unknown patient kind %d", kind);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // results are staged here and copied out only once every group has
    // succeeded, so that a failing call writes no output
    std::vector<dbq_hit> staged((size_t)nq * (size_t)(k > 0 ? k : 0));
    std::vector<const dbq_db*> owner((size_t)nq, nullptr);
    // group queries by database, keeping their order inside a group
    std::vector<int> order((size_t)nq);
    for (int q = 0; q < nq; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return db_of_query[a] < db_of_query[b]; });
    size_t i = 0;
    while (i < order.size()) {
        const int dbi = db_of_query[order[i]];
        size_t j = i;
        while (j < order.size() && db_of_query[order[j]] == dbi) ++j;
        dbq_db* db = dbs[dbi];
        if (!db) return fail(DBQ_EINVAL, "database %d is NULL", dbi);
        std::lock_guard<std::mutex> lock(db->mu);
        if (db->ds_factor)
            return fail(DBQ_ESTATE, "downsampled databases take single-patient queries only");
        DeviceGuard guard(db->device);
        if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
        for (size_t g0 = i; g0 < j; g0 += kBatchQ) {
            const int gn = (int)std::min<size_t>(kBatchQ, j - g0);
            float a1 = t1 ? t1[order[g0]] : NAN, a2 = t2 ? t2[order[g0]] : NAN;
            int rc = check_query_args(db, kind, &a1, &a2, k);
            if (rc) return rc;
            rc = ensure_batch(db, k);
            if (rc) return rc;
            if (mode == DBQ_MODE_EXACT) {
                for (int q = 0; q < gn; ++q) {
                    const int qi = order[g0 + q];
                    float b1 = t1 ? t1[qi] : NAN, b2 = t2 ? t2[qi] : NAN;
                    rc = check_query_args(db, kind, &b1, &b2, k);
                    if (!rc) rc = prepare_patient(db, patients[qi], kind, b1, b2, s);
                    if (!rc) rc = launch_query(db, k, db->bhits + (size_t)q * k, nullptr, s);
                    if (rc) return rc;
                }
            } else {
                if (db->storage != DBQ_STORE_BITS)
                    return fail(DBQ_EINVAL, "embedding modes need a bit-packed database");
                rc = check_prefilter_args(db, mode, n_candidates, k);
                if (rc) return rc;
                std::vector<const void*> pp((size_t)gn);
                for (int q = 0; q < gn; ++q) {
                    const int qi = order[g0 + q];
                    float b1 = t1 ? t1[qi] : NAN, b2 = t2 ? t2[qi] : NAN;
                    rc = check_query_args(db, kind, &b1, &b2, k);
                    if (rc) return rc;
                    pp[q] = patients[qi];
                }
                mark(db, 0, s);
                rc = prepare_batch(db, gn, pp.data(), kind, db->t1, db->t2, s);
                if (!rc) rc = run_prefilter(db, gn, mode, n_candidates, s);
                if (rc) return rc;
                dbq::RerankArgs r;
                r.planes = reinterpret_cast<const uint4*>(db->planes);
                r.ecount = db->ecount;
                r.n = db->n;
                r.wp4 = db->wp4;
                r.chunk4 = db->chunk4;
                r.nchunks = db->nchunks;
                r.patients = reinterpret_cast<const uint4*>(db->bplanes);
                r.pcounts = db->bpcount;
                r.cand = db->bcand;
                r.nq = gn;
                r.c = n_candidates;
                r.k = k;
                r.slices = rerank_slices(gn, n_candidates, db->grid);
                r.scratch = db->brr;
                r.tickets = db->btickets;
                r.hits = db->bhits;
                r.sup_lists = db->sparse ? db->bsup : nullptr;
                r.sup_lens = db->sparse ? db->bsuplen : nullptr;
                r.sched = db->sparse ? db->btickets + kBatchQ : nullptr;
                // a dense batch of kRerankDedupeMinQ queries or more reads each
                // distinct candidate once (DBQ_OPT_RERANK 2: every dense batch;
                // 1: none)
                const bool dedupe =
                    !db->sparse && (db->rerank_mode == 2 ||
                                    (db->rerank_mode == 0 && gn >= kRerankDedupeMinQ));
                if (dedupe) {
                    rc = ensure_rerank_partial(db, (int64_t)gn * n_candidates);
                    if (rc) return rc;
                }
                cudaError_t err = dedupe ? dbq::launch_rerank_dedupe(r, db->rrd, s)
                                         : dbq::launch_rerank(r, s);
                if (err != cudaSuccess) return cuda_fail(err, "re-rank launch");
                mark(db, 5, s);
                db->ev_valid = db->ev[0] != nullptr;
            }
            DBQ_CUDA(cudaMemcpyAsync(db->bhits_host, db->bhits, (size_t)gn * k * sizeof(dbq::Hit),
                                     cudaMemcpyDeviceToHost, s));
            if (mode != DBQ_MODE_EXACT) {
                rc = check_status(db, s);
                if (rc) return rc;
            }
            DBQ_CUDA(cudaStreamSynchronize(s));
            for (int q = 0; q < gn; ++q) {
                const int qi = order[g0 + q];
                const dbq_hit* got = reinterpret_cast<const dbq_hit*>(db->bhits_host) + (size_t)q * k;
                for (int h = 0; h < k; ++h)
                    if (got[h].index < 0 || got[h].index >= db->n)
                        return fail(DBQ_ECUDA, "kernel returned index %lld",
                                    (long long)got[h].index);
                std::memcpy(&staged[(size_t)qi * k], got, (size_t)k * sizeof(dbq_hit));
                owner[(size_t)qi] = db;
            }
        }
        i = j;
    }
    if (nq > 0) std::memcpy(hits, staged.data(), staged.size() * sizeof(dbq_hit));
    for (int qi = 0; qi < nq && params; ++qi) {
        const dbq_db* db = owner[(size_t)qi];
        for (int h = 0; h < k && db->n_params; ++h)
            std::memcpy(params + ((size_t)qi * k + h) * db->n_params,
                        &db->params[(size_t)staged[(size_t)qi * k + h].index * db->n_params],
                        sizeof(double) * db->n_params);
    }
    return DBQ_OK;
}

int db_set_option(dbq_db* db, int option, int64_t value)
{
    if (!db) return fail(DBQ_EINVAL, "db is NULL");
    std::lock_guard<std::mutex> lock(db->mu);
    if (option == DBQ_OPT_SPARSE) {
        if (value < 0 || value > 2) return fail(DBQ_EINVAL, "DBQ_OPT_SPARSE takes 0, 1 or 2");
        if (value == 2) {
            if (db->storage != DBQ_STORE_BITS)
                return fail(DBQ_EINVAL, "the word-major sparse scan needs bit-packed storage");
            if (!db->planes_t) {
                DeviceGuard guard(db->device);
                if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
                int rc = dev_alloc(db, &db->planes_t, (size_t)db->n * 2 * db->wp * 4,
                                   "word-major planes");
                if (!rc) rc = dev_alloc(db, &db->tcounts, (size_t)db->n * 2 * 4,
                                        "word-major sparse counts");
                if (rc) {
                    if (db->planes_t) db->bytes_held -= (size_t)db->n * 2 * db->wp * 4;
                    cudaFree(db->planes_t);
                    db->planes_t = nullptr;
                    return rc;
                }
                db->planes_t_valid = false;
            }
            if (db->built && !db->planes_t_valid) {   // built now, not at the first scan
                DeviceGuard guard(db->device);
                if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", db->device);
                cudaError_t err = dbq::launch_transpose_planes(
                    reinterpret_cast<const uint4*>(db->planes), db->n, 2 * (int)db->wp4,
                    db->planes_t, nullptr);
                if (err == cudaSuccess) err = cudaStreamSynchronize(nullptr);
                if (err != cudaSuccess) return cuda_fail(err, "word-major copy");
                db->planes_t_valid = true;
            }
        }
        db->sparse = value != 0;
        db->sparse_mode = (int)value;
        db->prepared = false;   // a prepared patient has no support lists yet
        return DBQ_OK;
    }
    if (option == DBQ_OPT_RERANK) {
        if (value < 0 || value > 2) return fail(DBQ_EINVAL, "DBQ_OPT_RERANK takes 0, 1 or 2");
        db->rerank_mode = (int)value;
        return DBQ_OK;
    }
    return fail(DBQ_EINVAL, "unknown option %d", option);
}

int db_last_support(dbq_db* db, int64_t out[2])
{
    if (!db || !out) return fail(DBQ_EINVAL, "NULL pointer argument");
    std::lock_guard<std::mutex> lock(db->mu);
    if (!db->sparse || !db->prepared || db->storage != DBQ_STORE_BITS)
        return fail(DBQ_ESTATE, "no sparse patient prepared");
    DeviceGuard guard(db->device);
    uint32_t len[2] = {0, 0};
    DBQ_CUDA(cudaMemcpy(len, db->plen, sizeof len, cudaMemcpyDeviceToHost));
    out[0] = len[0];
    out[1] = len[1];
    return DBQ_OK;
}

int db_stage_times(dbq_db* db, float* ms, int n)
{
    if (!db || !ms) return fail(DBQ_EINVAL, "NULL pointer argument");
    std::lock_guard<std::mutex> lock(db->mu);
    if (!db->ev_valid) return fail(DBQ_ESTATE, "no embedding batch has run on this handle");
    DeviceGuard guard(db->device);
    for (int i = 0; i < n && i < 5; ++i) {
        float t = 0.f;
        DBQ_CUDA(cudaEventElapsedTime(&t, db->ev[i], db->ev[i + 1]));
        ms[i] = t;
    }
    return DBQ_OK;
}

int db_plan_create(dbq_plan** out, dbq_db* const* dbs, int ndb, int max_queries, int k)
{
    if (!out || !dbs) return fail(DBQ_EINVAL, "NULL pointer argument");
    *out = nullptr;
    if (ndb < 1 || max_queries < 1 || max_queries > 65535)
        return fail(DBQ_EINVAL, "need 1 <= ndb and 1 <= max_queries <= 65535");
    if (k < 1 || k > kMaxK) return fail(DBQ_ERANGE, "k must be in [1, %d]", kMaxK);
    dbq_plan* p = new (std::nothrow) dbq_plan;
    if (!p) return fail(DBQ_ENOMEM, "host allocation failed");
    p->maxq = max_queries;
    p->k = k;
    for (int i = 0; i < ndb; ++i) {
        dbq_db* db = dbs[i];
        if (!db) { delete p; return fail(DBQ_EINVAL, "database %d is NULL", i); }
        std::lock_guard<std::mutex> lock(db->mu);
        if (db->storage != DBQ_STORE_BITS || !db->built || db->ds_factor) {
            delete p;
            return fail(DBQ_ESTATE,
                        "plans need built full-resolution bit-packed databases (database %d)", i);
        }
        if (i == 0) p->device = db->device;
        if (db->device != p->device) {
            delete p;
            return fail(DBQ_EINVAL, "all databases of a plan must be on one device");
        }
        if (k > db->n) { delete p; return fail(DBQ_ERANGE, "k exceeds database %d size", i); }
        p->max_wp = std::max<int64_t>(p->max_wp, db->wp);
        p->dbs.push_back(db);
    }
    DeviceGuard guard(p->device);
    if (!guard.ok) { delete p; return fail(DBQ_ECUDA, "cannot select device"); }
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
    const size_t q = (size_t)max_queries;
    const size_t max_items = q * p->max_slices;
    auto dalloc = [&](auto** ptr, size_t bytes) -> bool {
        if (cudaMalloc(reinterpret_cast<void**>(ptr), bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            *ptr = nullptr;
            return false;
        }
        return true;
    };
    auto halloc = [&](auto** ptr, size_t bytes) -> bool {
        if (cudaMallocHost(reinterpret_cast<void**>(ptr), bytes) != cudaSuccess) {
            cudaGetLastError();
            *ptr = nullptr;
            return false;
        }
        return true;
    };
    bool ok = dalloc(&p->planes, q * 2 * p->max_wp * 4) && dalloc(&p->pcount, q * 2 * 4) &&
              dalloc(&p->sup, q * 2 * (p->max_wp / 4) * 4) && dalloc(&p->suplen, q * 2 * 4) &&
              dalloc(&p->scratch, q * p->max_slices * k * sizeof(dbq::Cand)) &&
              dalloc(&p->tickets, q * 4) && dalloc(&p->counter, 16) &&
              dalloc(&p->tasks_dev, q * sizeof(dbq::QueryTask)) &&
              halloc(&p->tasks_host, q * sizeof(dbq::QueryTask)) &&
              dalloc(&p->items_dev, max_items * sizeof(int2)) &&
              halloc(&p->items_host, max_items * sizeof(int2)) &&
              dalloc(&p->ptrs_dev, q * sizeof(void*)) && halloc(&p->ptrs_host, q * sizeof(void*));
    if (!ok) {
        delete p;
        return fail(DBQ_ENOMEM, "plan allocation failed");
    }
    // counts of the tensor-core path: at most 1 GiB, for 16 to 128 queries
    // per launch; databases beyond 2^24 voxels stay on the CUDA-core path
    int64_t tc_n = 0;
    for (const dbq_db* db : p->dbs)
        if (db->v <= (int64_t)1 << 24) tc_n = std::max<int64_t>(tc_n, db->n);
    if (tc_n > 0) {
        const size_t row_bytes = (size_t)dbq::tc_counts_stride(tc_n) * 2 * sizeof(uint32_t);
        int rows = std::min(max_queries, dbq::tc_scan_max_queries());
        while (rows > 16 && (size_t)rows * row_bytes > ((size_t)1 << 30)) rows /= 2;
        if ((size_t)rows * row_bytes <= ((size_t)1 << 30) &&
            dalloc(&p->tc_counts, (size_t)rows * row_bytes) &&
            dalloc(&p->tc_status, 16))
            p->tc_rows = rows;
        else
            cudaGetLastError();
    }
    cudaError_t err = cudaMemset(p->tickets, 0, q * 4);
    if (err == cudaSuccess && p->tc_status) err = cudaMemset(p->tc_status, 0, 16);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&p->copied, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        delete p;
        return cuda_fail(err, "plan initialisation");
    }
    *out = p;
    return DBQ_OK;
}

int db_plan_set(dbq_plan* plan, int param, int64_t value)
{
    if (!plan) return fail(DBQ_EINVAL, "plan is NULL");
    if (param == DBQ_PLAN_ITEMS_PER_SM) {
        if (value < 1 || value > 64) return fail(DBQ_EINVAL, "items per SM must be in [1, 64]");
        plan->items_per_sm = (int)value;
        return DBQ_OK;
    }
    if (param == DBQ_PLAN_TC_MIN_QUERIES) {
        if (value < 0 || value > 65535)
            return fail(DBQ_EINVAL, "tensor-core query threshold must be in [0, 65535]");
        plan->tc_min = (int)value;
        return DBQ_OK;
    }
    if (param == DBQ_PLAN_TEST_STALL_NS) {
        if (value < 0 || value > 2000000000LL)
            return fail(DBQ_EINVAL, "stall must be in [0, 2e9] ns");
        plan->tc_stall_ns = (unsigned long long)value;
        return DBQ_OK;
    }
    return fail(DBQ_EINVAL, "unknown plan parameter %d", param);
}

int db_plan_set_for(dbq_plan* plan, int db_index, int param, int64_t value)
{
    if (!plan) return fail(DBQ_EINVAL, "plan is NULL");
    if (db_index < 0 || db_index >= (int)plan->dbs.size())
        return fail(DBQ_ERANGE, "database index %d outside the plan", db_index);
    if (param != DBQ_PLAN_TC_MIN_QUERIES)
        return fail(DBQ_EINVAL, "plan parameter %d has no per-database value", param);
    if (value < -1 || value > 65535)
        return fail(DBQ_EINVAL, "tensor-core query threshold must be in [-1, 65535]");
    if (plan->tc_min_db.size() != plan->dbs.size()) plan->tc_min_db.assign(plan->dbs.size(), -1);
    plan->tc_min_db[(size_t)db_index] = (int)value;
    return DBQ_OK;
}

int db_plan_query(dbq_plan* p, const int* db_of_query, int nq, const void* const* patients_dev,
                  int kind, const float* t1, const float* t2, dbq_hit* hits_dev, void* stream)
{
    if (!p || !db_of_query || !patients_dev || !hits_dev)
        return fail(DBQ_EINVAL, "NULL pointer argument");
    if (nq < 1 || nq > p->maxq) return fail(DBQ_ERANGE, "nq must be in [1, %d]", p->maxq);
    if (kind != DBQ_F32 && kind != DBQ_F16 && kind != DBQ_BITS)
        return fail(DBQ_EINVAL, "unknown patient kind %d", kind);
    DeviceGuard guard(p->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", p->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    DBQ_CUDA(cudaStreamIsCapturing(s, &cap));
    if (p->copy_pending && cap == cudaStreamCaptureStatusNone) {
        DBQ_CUDA(cudaEventSynchronize(p->copied));   // host tables free for reuse
        p->copy_pending = false;
    }
    const int ndb = (int)p->dbs.size();
    for (int q = 0; q < nq; ++q) {
        const int d = db_of_query[q];
        if (d < 0 || d >= ndb) return fail(DBQ_EINVAL, "query %d names database %d", q, d);
        if (!patients_dev[q]) return fail(DBQ_EINVAL, "patient %d is NULL", q);
        dbq_db* db = p->dbs[d];
        float a = t1 ? t1[q] : NAN, b = t2 ? t2[q] : NAN;
        if ((!std::isnan(a) && a != db->t1) || (!std::isnan(b) && b != db->t2))
            return fail(DBQ_EINVAL, "query %d: thresholds differ from database %d's", q, d);
    }
    // group the queries by database; each group's patient slots are contiguous
    std::vector<int> order((size_t)nq);
    for (int q = 0; q < nq; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return db_of_query[a] < db_of_query[b]; });
    // databases whose dense queries go to the tensor-core contraction
    std::vector<int> per_db((size_t)ndb, 0);
    for (int q = 0; q < nq; ++q) ++per_db[db_of_query[q]];
    std::vector<char> use_tc((size_t)ndb, 0);
    for (int d = 0; d < ndb; ++d) {
        const dbq_db* db = p->dbs[d];
        const int thr = (size_t)d < p->tc_min_db.size() && p->tc_min_db[(size_t)d] >= 0
                            ? p->tc_min_db[(size_t)d] : p->tc_min;
        use_tc[d] = p->tc_rows > 0 && thr > 0 && per_db[d] >= thr &&
                    db->v <= ((int64_t)1 << 24) && db->wp >= dbq::tc_scan_min_words();
    }
    // databases with a word-major copy (DBQ_OPT_SPARSE 2) whose queries stay off
    // the contraction: counts of all their queries over the copy, then the
    // contraction's per-query selection on those counts
    std::vector<char> use_wm((size_t)ndb, 0);
    for (int d = 0; d < ndb; ++d) {
        const dbq_db* db = p->dbs[d];
        use_wm[d] = !use_tc[d] && p->tc_rows > 0 && db->sparse_mode == 2 && db->planes_t &&
                    db->planes_t_valid && db->v <= ((int64_t)1 << 24);
    }
    // work-item budget: items_per_sm * SMs, shared in proportion to bytes
    double total = 0;
    for (int q = 0; q < nq; ++q) {
        const dbq_db* db = p->dbs[db_of_query[q]];
        if (!use_tc[db_of_query[q]] && !use_wm[db_of_query[q]]) total += (double)db->n * db->wp4;
    }
    struct TcGroup {
        const dbq_db* db;
        int slot, cnt;
        const uint32_t* qplanes;
    };
    std::vector<TcGroup> tc_groups;
    struct WmGroup {
        const dbq_db* db;
        int slot, cnt;
        const uint32_t* qplanes;
        const uint32_t* sup;
        const uint32_t* len;
    };
    std::vector<WmGroup> wm_groups;
    const double budget = (double)p->items_per_sm * p->sms;
    int nitems = 0;
    size_t word_off = 0, sup_off = 0;
    int slot = 0;
    size_t g = 0;
    while (g < order.size()) {
        const int d = db_of_query[order[g]];
        size_t h = g;
        while (h < order.size() && db_of_query[order[h]] == d) ++h;
        dbq_db* db = p->dbs[d];
        const int cnt = (int)(h - g);
        uint32_t* gplanes = p->planes + word_off;
        uint32_t* gcount = p->pcount + 2 * slot;
        uint32_t* gsup = p->sup + sup_off;
        uint32_t* glen = p->suplen + 2 * slot;
        DBQ_CUDA(cudaMemsetAsync(gcount, 0, (size_t)cnt * 2 * 4, s));
        if (kind == DBQ_BITS) {
            for (int i = 0; i < cnt; ++i) {
                cudaError_t err = dbq::launch_import_bits(
                    static_cast<const uint32_t*>(patients_dev[order[g + i]]), db->words, db->v,
                    db->wp, gplanes + (size_t)i * 2 * db->wp, gcount + 2 * i, s);
                if (err != cudaSuccess) return cuda_fail(err, "patient import");
            }
        } else {
            for (int i = 0; i < cnt; ++i) p->ptrs_host[slot + i] = patients_dev[order[g + i]];
            DBQ_CUDA(cudaMemcpyAsync(p->ptrs_dev + slot, p->ptrs_host + slot,
                                     (size_t)cnt * sizeof(void*), cudaMemcpyHostToDevice, s));
            cudaError_t err = dbq::launch_pack_ptrs(p->ptrs_dev + slot, kind == DBQ_F16, cnt,
                                                    db->v, db->wp, db->t1, db->t2, gplanes,
                                                    gcount, s);
            if (err != cudaSuccess) return cuda_fail(err, "patient packing");
        }
        if (db->sparse) {
            cudaError_t err = dbq::launch_support(gplanes, cnt, db->wp4, gsup, glen, s);
            if (err != cudaSuccess) return cuda_fail(err, "support list launch");
        }
        for (int i = 0; i < cnt; ++i) {
            const int q = order[g + i];
            dbq::QueryTask& t = p->tasks_host[slot + i];
            t.planes = reinterpret_cast<const uint4*>(db->planes);
            t.ecount = db->ecount;
            t.n = db->n;
            t.wp4 = db->wp4;
            t.chunk4 = db->chunk4;
            t.nchunks = db->nchunks;
            t.k = p->k;
            int sl = 1;
            if (!use_tc[d] && !use_wm[d] && total > 0)
                sl = (int)std::lround(budget * ((double)db->n * db->wp4) / total);
            sl = std::max(1, std::min(sl, p->max_slices));
            if ((int64_t)sl > db->n) sl = (int)db->n;
            t.slices = sl;
            t.patient = reinterpret_cast<const uint4*>(gplanes + (size_t)i * 2 * db->wp);
            t.pcount = gcount + 2 * i;
            t.sup_list = db->sparse ? gsup + (size_t)i * 2 * db->wp4 : nullptr;
            t.sup_len = db->sparse ? glen + 2 * i : nullptr;
            t.scratch = p->scratch + (size_t)(slot + i) * p->max_slices * p->k;
            t.ticket = p->tickets + slot + i;
            t.hits = reinterpret_cast<dbq::Hit*>(hits_dev) + (size_t)q * p->k;
        }
        if (use_tc[d]) {
            // no work items: the group runs as a contraction after the scan
            for (int i = 0; i < cnt; ++i) p->tasks_host[slot + i].slices = 0;
            tc_groups.push_back({db, slot, cnt, gplanes});
        } else if (use_wm[d]) {
            // no work items: counts over the word-major copy after the scan
            for (int i = 0; i < cnt; ++i) p->tasks_host[slot + i].slices = 0;
            wm_groups.push_back({db, slot, cnt, gplanes, gsup, glen});
        } else {
            // slice-major: the same entry slice of every query of this
            // database in consecutive items, so CTAs that run them at the
            // same time read those entries from HBM once and share them
            // through L2
            const int gsl = p->tasks_host[slot].slices;      // equal within a database
            for (int j = 0; j < gsl; ++j)
                for (int i = 0; i < cnt; ++i) p->items_host[nitems++] = make_int2(slot + i, j);
        }
        word_off += (size_t)cnt * 2 * db->wp;
        sup_off += (size_t)cnt * 2 * db->wp4;
        slot += cnt;
        g = h;
    }
    DBQ_CUDA(cudaMemcpyAsync(p->tasks_dev, p->tasks_host, (size_t)nq * sizeof(dbq::QueryTask),
                             cudaMemcpyHostToDevice, s));
    DBQ_CUDA(cudaMemcpyAsync(p->items_dev, p->items_host, (size_t)nitems * sizeof(int2),
                             cudaMemcpyHostToDevice, s));
    if (cap == cudaStreamCaptureStatusNone) {
        DBQ_CUDA(cudaEventRecord(p->copied, s));
        p->copy_pending = true;
    }
    bool any_sparse = false;
    for (int q = 0; q < nq; ++q) any_sparse |= p->dbs[db_of_query[q]]->sparse;
    cudaError_t err = dbq::launch_scan_tasks(p->tasks_dev, nq, p->items_dev, nitems, p->counter,
                                             p->sms, any_sparse, s);
    if (err != cudaSuccess) return cuda_fail(err, "task scan launch");
    for (const TcGroup& tg : tc_groups) {
        for (int c0 = 0; c0 < tg.cnt; c0 += p->tc_rows) {
            const int nqc = std::min(p->tc_rows, tg.cnt - c0);
            dbq::TcScanArgs ta;
            ta.planes = tg.db->planes;
            ta.n = tg.db->n;
            ta.wp = tg.db->wp;
            ta.qplanes = tg.qplanes + (size_t)c0 * 2 * tg.db->wp;
            ta.nq = nqc;
            ta.counts = p->tc_counts;
            ta.stride = dbq::tc_counts_stride(tg.db->n);
            ta.status = p->tc_status;
            ta.stall_ns = p->tc_stall_ns;
            err = dbq::launch_tc_scan(ta, p->sms, s);
            if (err != cudaSuccess) return cuda_fail(err, "tensor-core scan launch");
            err = dbq::launch_tc_select(p->tasks_dev, tg.slot + c0, nqc, p->tc_counts, tg.db->n,
                                        ta.stride, s);
            if (err != cudaSuccess) return cuda_fail(err, "tensor-core selection launch");
        }
    }
    for (const WmGroup& wg : wm_groups) {
        const int64_t stride = dbq::tc_counts_stride(wg.db->n);
        for (int c0 = 0; c0 < wg.cnt; c0 += p->tc_rows) {
            const int nqc = std::min(p->tc_rows, wg.cnt - c0);
            DBQ_CUDA(cudaMemsetAsync(p->tc_counts, 0, (size_t)2 * nqc * stride * 4, s));
            err = dbq::launch_sparse_t_count(
                wg.db->planes_t, wg.db->n, nqc,
                reinterpret_cast<const uint4*>(wg.qplanes + (size_t)c0 * 2 * wg.db->wp),
                (int)wg.db->wp4, wg.sup + (size_t)c0 * 2 * wg.db->wp4, wg.len + 2 * c0,
                p->tc_counts, stride, 1, (int64_t)nqc * stride, p->sms, s);
            if (err != cudaSuccess) return cuda_fail(err, "word-major sparse count launch");
            err = dbq::launch_tc_select(p->tasks_dev, wg.slot + c0, nqc, p->tc_counts, wg.db->n,
                                        stride, s);
            if (err != cudaSuccess) return cuda_fail(err, "selection launch");
        }
    }
    return DBQ_OK;
}

int db_plan_status(dbq_plan* p, void* stream)
{
    if (!p) return fail(DBQ_EINVAL, "plan is NULL");
    DeviceGuard guard(p->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", p->device);
    if (!p->tc_status) return DBQ_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int st = 0;
    DBQ_CUDA(cudaMemcpyAsync(&st, p->tc_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    DBQ_CUDA(cudaStreamSynchronize(s));
    if (st != 0) {
        DBQ_CUDA(cudaMemsetAsync(p->tc_status, 0, sizeof(int), s));
        DBQ_CUDA(cudaStreamSynchronize(s));
        return fail(DBQ_ETIMEOUT, "a tensor-core wait timed out (code %d)", st);
    }
    return DBQ_OK;
}

int db_plan_destroy(dbq_plan* plan)
{
    if (!plan) return DBQ_OK;
    DeviceGuard guard(plan->device);
    cudaDeviceSynchronize();
    delete plan;
    return DBQ_OK;
}

int db_info(const dbq_db* db, int64_t out[8])
{
    if (!db || !out) return fail(DBQ_EINVAL, "NULL pointer argument");
    out[0] = db->n;
    out[1] = db->v;
    out[2] = db->words;
    out[3] = db->wp;
    out[4] = db->storage;
    out[5] = db->built ? 1 : 0;
    out[6] = db->n_params;
    out[7] = (int64_t)db->bytes_held;
    return DBQ_OK;
}

int db_destroy(dbq_db* db)
{
    if (!db) return DBQ_OK;
    {
        DeviceGuard guard(db->device);
        cudaDeviceSynchronize();
        delete db;
    }
    return DBQ_OK;
}

int rd_create(rd_solver** out, int nx, int ny, int nz, const float* tissue, int batch)
{
    if (!out) return fail(DBQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(DBQ_EINVAL, "grid dimensions must be >= 1");
    const int64_t v = (int64_t)nx * ny * nz;
    if (v >= (int64_t(1) << 31)) return fail(DBQ_EINVAL, "grid too large");
    if (!tissue) return fail(DBQ_EINVAL, "tissue is NULL");
    if (batch == 0) batch = 16;
    if (batch < 1 || batch > 1024) return fail(DBQ_EINVAL, "batch must be in [1, 1024]");
    int dev = 0;
    DBQ_CUDA(cudaGetDevice(&dev));
    rd_solver* rs = new (std::nothrow) rd_solver;
    if (!rs) return fail(DBQ_ENOMEM, "host allocation failed");
    rs->device = dev;
    rs->nx = nx;
    rs->ny = ny;
    rs->nz = nz;
    rs->v = v;
    rs->batch = batch;
    try {
        rs->tissue.resize((size_t)v);
    } catch (...) {
        delete rs;
        return fail(DBQ_ENOMEM, "host allocation of the tissue copy failed");
    }
    cudaError_t err = cudaMemcpy(rs->tissue.data(), tissue, (size_t)v * 4, cudaMemcpyDefault);
    if (err != cudaSuccess) {
        delete rs;
        return cuda_fail(err, "tissue copy");
    }
    for (int64_t i = 0; i < v; ++i) {
        const float m = rs->tissue[(size_t)i];
        if (!(m >= 0.0f) || !std::isfinite(m)) {
            delete rs;
            return fail(DBQ_EINVAL, "tissue value %lld is negative or not finite", (long long)i);
        }
        rs->m_max = std::max(rs->m_max, (double)m);
    }
    int rc = rd_alloc(&rs->m_dev, (size_t)v * 4, "tissue map");
    if (!rc) rc = rd_alloc(&rs->hx, (size_t)v * 4, "x faces");
    if (!rc) rc = rd_alloc(&rs->hy, (size_t)v * 4, "y faces");
    if (!rc) rc = rd_alloc(&rs->hz, (size_t)v * 4, "z faces");
    if (!rc) rc = rd_alloc(&rs->hym, (size_t)v * 4, "-y faces");
    if (!rc) rc = rd_alloc(&rs->tile_any, (size_t)dbq::rd_tiles(nx, ny, nz) * 4, "tile flags");
    if (!rc) rc = rd_alloc(&rs->sims, (size_t)batch * sizeof(dbq::RdSim), "simulation table");
    if (!rc) rc = rd_alloc(&rs->buf0, (size_t)batch * v * 4, "fields (even steps)");
    if (!rc) rc = rd_alloc(&rs->buf1, (size_t)batch * v * 4, "fields (odd steps)");
    if (!rc) rc = rd_alloc(&rs->updates, sizeof(unsigned long long), "update counter");
    if (rc) {
        delete rs;
        return rc;
    }
    err = cudaMemcpy(rs->m_dev, rs->tissue.data(), (size_t)v * 4, cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = dbq::launch_rd_faces(rs->m_dev, nx, ny, nz, rs->hx, rs->hy, rs->hz, rs->hym,
                                   rs->tile_any, nullptr);
    if (err == cudaSuccess) err = cudaEventCreate(&rs->ev0);
    if (err == cudaSuccess) err = cudaEventCreate(&rs->ev1);
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        delete rs;
        return cuda_fail(err, "face coefficients");
    }
    *out = rs;
    return DBQ_OK;
}

int rd_simulate(rd_solver* rs, int count, const double* theta, float u0, double cfl,
                float* out, int64_t* steps, void* stream)
{
    if (!rs) return fail(DBQ_EINVAL, "solver is NULL");
    std::lock_guard<std::mutex> lock(rs->mu);
    if (count < 0) return fail(DBQ_EINVAL, "count < 0");
    if (count == 0) return DBQ_OK;
    if (!theta || !out) return fail(DBQ_EINVAL, "NULL pointer argument");
    if (!(u0 > 0.0f && u0 <= 1.0f)) return fail(DBQ_EINVAL, "u0 must be in (0, 1]");
    if (!(cfl > 0.0 && cfl <= 1.0)) return fail(DBQ_EINVAL, "cfl must be in (0, 1]");
    std::vector<dbq::RdSim> sims((size_t)count);
    for (int j = 0; j < count; ++j) {
        const double* t = theta + (size_t)j * 6;
        for (int q = 0; q < 6; ++q)
            if (!std::isfinite(t[q])) return fail(DBQ_EINVAL, "theta[%d] is not finite", j);
        if (t[3] < 0.0 || t[4] < 0.0 || t[5] < 0.0)
            return fail(DBQ_EINVAL, "theta[%d]: D_w, rho and T_end must be >= 0", j);
        const double fx = std::floor(t[0] + 0.5), fy = std::floor(t[1] + 0.5),
                     fz = std::floor(t[2] + 0.5);
        if (fx < 0 || fy < 0 || fz < 0 || fx >= rs->nx || fy >= rs->ny || fz >= rs->nz)
            return fail(DBQ_EINVAL, "theta[%d]: seed outside the grid", j);
        const int64_t seed = (int64_t)fx + (int64_t)rs->nx * ((int64_t)fy + (int64_t)rs->ny * (int64_t)fz);
        if (!(rs->tissue[(size_t)seed] > 0.0f))
            return fail(DBQ_EINVAL, "theta[%d]: seed outside the domain (tissue 0)", j);
        const int64_t n = rd_step_count(t[5], t[3], t[4], rs->m_max, cfl);
        if (n > 0x7fffffff) return fail(DBQ_EINVAL, "theta[%d]: too many steps", j);
        const double dt = n ? t[5] / (double)n : 0.0;
        dbq::RdSim& p = sims[(size_t)j];
        p.a = (float)(dt * t[3]);
        p.b = (float)(dt * t[4]);
        p.steps = (int32_t)n;
        p.sx = (int32_t)fx;
        p.sy = (int32_t)fy;
        p.sz = (int32_t)fz;
        p.start = 0;
    }
    DeviceGuard guard(rs->device);
    if (!guard.ok) return fail(DBQ_ECUDA, "cannot select device %d", rs->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // Continuous batching over `slots` slots: longest simulations first, a
    // slot is refilled (fields zeroed, seed set, table entry replaced) in
    // stream order right after the launch that ends its simulation.
    std::vector<int> order((size_t)count);
    for (int j = 0; j < count; ++j) order[(size_t)j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return sims[(size_t)x].steps > sims[(size_t)y].steps;
    });
    const int slots = std::min(rs->batch, count);
    std::vector<dbq::RdSim> table((size_t)slots);
    std::vector<int> slot_sim((size_t)slots, -1);
    for (dbq::RdSim& e : table) e = dbq::RdSim{0.f, 0.f, 0, 0, 0, 0, 0};
    size_t next = 0;
    int launch = 0;
    const size_t vbytes = (size_t)rs->v * 4;
    auto copy_out = [&](int sl) -> cudaError_t {
        const dbq::RdSim& e = table[(size_t)sl];
        const float* src = (e.steps & 1 ? rs->buf1 : rs->buf0) + (size_t)sl * rs->v;
        return cudaMemcpyAsync(out + (size_t)slot_sim[(size_t)sl] * rs->v, src, vbytes,
                               cudaMemcpyDefault, s);
    };
    // put the next simulation with steps > 0 in slot sl (those with none are
    // their initial condition: seeded and copied out at once)
    auto fill = [&](int sl) -> cudaError_t {
        table[(size_t)sl].steps = 0;
        slot_sim[(size_t)sl] = -1;
        while (next < order.size()) {
            const int j = order[next++];
            dbq::RdSim e = sims[(size_t)j];
            e.start = launch;
            float* b0 = rs->buf0 + (size_t)sl * rs->v;
            cudaError_t err = cudaMemsetAsync(b0, 0, vbytes, s);
            if (err == cudaSuccess)
                err = cudaMemsetAsync(rs->buf1 + (size_t)sl * rs->v, 0, vbytes, s);
            const int64_t seed = e.sx + (int64_t)rs->nx * (e.sy + (int64_t)rs->ny * e.sz);
            if (err == cudaSuccess)
                err = cudaMemcpyAsync(b0 + seed, &u0, sizeof(float), cudaMemcpyHostToDevice, s);
            if (err != cudaSuccess) return err;
            table[(size_t)sl] = e;
            slot_sim[(size_t)sl] = j;
            if (e.steps > 0) return cudaSuccess;
            err = copy_out(sl);
            if (err != cudaSuccess) return err;
            table[(size_t)sl].steps = 0;
            slot_sim[(size_t)sl] = -1;
        }
        return cudaSuccess;
    };
    dbq::RdStepArgs g;
    g.sims = rs->sims;
    g.hx = rs->hx;
    g.hy = rs->hy;
    g.hz = rs->hz;
    g.hym = rs->hym;
    g.tile_any = rs->tile_any;
    g.buf0 = rs->buf0;
    g.buf1 = rs->buf1;
    g.updates = rs->updates;
    g.nx = rs->nx;
    g.ny = rs->ny;
    g.nz = rs->nz;
    DBQ_CUDA(cudaMemsetAsync(rs->updates, 0, sizeof(unsigned long long), s));
    DBQ_CUDA(cudaEventRecord(rs->ev0, s));
    for (int sl = 0; sl < slots; ++sl) {
        cudaError_t err = fill(sl);
        if (err != cudaSuccess) return cuda_fail(err, "slot fill");
    }
    DBQ_CUDA(cudaMemcpyAsync(rs->sims, table.data(), (size_t)slots * sizeof(dbq::RdSim),
                             cudaMemcpyHostToDevice, s));
    for (;;) {
        bool busy = false;
        for (const dbq::RdSim& e : table) busy |= e.steps > 0;
        if (!busy) break;
        cudaError_t err = dbq::launch_rd_step(g, slots, launch, s);
        if (err != cudaSuccess) return cuda_fail(err, "step launch");
        ++launch;
        bool changed = false;
        for (int sl = 0; sl < slots; ++sl) {
            const dbq::RdSim& e = table[(size_t)sl];
            if (e.steps > 0 && e.start + e.steps == launch) {
                err = copy_out(sl);
                if (err == cudaSuccess) err = fill(sl);
                if (err != cudaSuccess) return cuda_fail(err, "slot refill");
                changed = true;
            }
        }
        if (changed)
            DBQ_CUDA(cudaMemcpyAsync(rs->sims, table.data(), (size_t)slots * sizeof(dbq::RdSim),
                                     cudaMemcpyHostToDevice, s));
    }
    DBQ_CUDA(cudaEventRecord(rs->ev1, s));
    unsigned long long updates = 0;
    DBQ_CUDA(cudaMemcpyAsync(&updates, rs->updates, sizeof updates, cudaMemcpyDeviceToHost, s));
    DBQ_CUDA(cudaStreamSynchronize(s));
    float ms = 0.0f;
    DBQ_CUDA(cudaEventElapsedTime(&ms, rs->ev0, rs->ev1));
    if (steps)
        for (int j = 0; j < count; ++j) steps[j] = sims[(size_t)j].steps;
    rs->stats[0] = ms;
    rs->stats[1] = launch;
    rs->stats[2] = (double)updates;
    rs->stats[3] = slots;
    rs->ran = true;
    return DBQ_OK;
}

int rd_stats(const rd_solver* rs, double out[4])
{
    if (!rs || !out) return fail(DBQ_EINVAL, "NULL pointer argument");
    if (!rs->ran) return fail(DBQ_ESTATE, "no simulation has run on this solver");
    for (int i = 0; i < 4; ++i) out[i] = rs->stats[i];
    return DBQ_OK;
}

int rd_destroy(rd_solver* rs)
{
    if (!rs) return DBQ_OK;
    DeviceGuard guard(rs->device);
    cudaDeviceSynchronize();
    delete rs;
    return DBQ_OK;
}

}  // extern "C"
