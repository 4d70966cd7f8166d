// lc_api.cu -- the C ABI declared in include/lc.h: argument checks, column
// ownership, the LCF1 header and directories, and host-side validation of
// serialized blobs.  Every compute step runs in the kernels of lc_compress.cu
// and lc_query.cu.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lc_internal.h"

namespace lcx {

static std::atomic<uint64_t> g_launches{0};

void note_launch(uint32_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {
std::atomic<bool> g_timing{false};
std::mutex g_timing_mu;
struct TimedLaunch {
    std::string name;
    cudaEvent_t a, b;
};
std::vector<TimedLaunch> g_timed;
std::map<std::string, std::pair<uint64_t, double>> g_totals;
}  // namespace

KTime::KTime(const char* n, cudaStream_t s) : name(n), st(s), a(nullptr), b(nullptr) {
    if (!g_timing.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        a = b = nullptr;
        return;
    }
    cudaEventRecord(a, st);
}

KTime::~KTime() {
    if (!a) return;
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_timed.push_back(TimedLaunch{name, a, b});
}

static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

HTime::HTime(const char* n) : name(n), t0(g_timing.load(std::memory_order_relaxed) ? now_ms() : -1.0) {}

HTime::~HTime() {
    if (t0 < 0) return;
    const double dt = now_ms() - t0;
    std::lock_guard<std::mutex> lk(g_timing_mu);
    auto& e = g_totals[std::string("host:") + name];
    e.first += 1;
    e.second += dt;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return LC_OK;
    if (e == cudaErrorMemoryAllocation) return LC_ERR_NOMEM;
    return LC_ERR_CUDA;
}

// ------------------------------------------------------------------ small transfers without copy engines

namespace {

constexpr size_t kStageCap = 8u << 20;  // per host thread and device
constexpr int kStageDevices = 64;

struct StageArena {
    uint8_t* h = nullptr;  // page-locked, mapped
    uint8_t* d = nullptr;  // its device address
    size_t off = 0;        // bytes in use since the last stage_sync
};
thread_local StageArena t_stage[kStageDevices];

__global__ void stage_copy16(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
__global__ void stage_copy1(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

int stage_arena(StageArena** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kStageDevices) return LC_ERR_INTERNAL;
    StageArena& a = t_stage[dev];
    if (!a.h) {
        void* h = nullptr;
        if (cudaHostAlloc(&h, kStageCap, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
            return LC_ERR_NOMEM;
        void* d = nullptr;
        if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
            cudaFreeHost(h);
            return LC_ERR_CUDA;
        }
        a.h = (uint8_t*)h;
        a.d = (uint8_t*)d;
        a.off = 0;
    }
    *out = &a;
    return LC_OK;
}

// A region of `bytes` (16-byte aligned); when the arena is full, waits for st
// (every region in use belongs to a transfer ordered on st before this one).
int stage_reserve(size_t bytes, cudaStream_t st, StageArena** arena, size_t* off) {
    if (bytes > kStageCap) return LC_ERR_UNSUPPORTED;
    StageArena* a = nullptr;
    int rc = stage_arena(&a);
    if (rc) return rc;
    if (a->off + bytes > kStageCap) {
        rc = cuda_status(cudaStreamSynchronize(st));
        if (rc) return rc;
        a->off = 0;
    }
    *arena = a;
    *off = a->off;
    a->off = (a->off + bytes + 15) & ~(size_t)15;
    return LC_OK;
}

int stage_copy(const uint8_t* src, uint8_t* dst, size_t bytes, cudaStream_t st) {
    const bool v16 = ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
    const size_t n16 = v16 ? bytes / 16 : 0, tail = bytes - 16 * n16;
    if (n16) {
        stage_copy16<<<(unsigned)std::min<size_t>((n16 + 255) / 256, 1024), 256, 0, st>>>((const uint4*)src,
                                                                                           (uint4*)dst, n16);
        note_launch();
    }
    if (tail) {
        stage_copy1<<<(unsigned)std::min<size_t>((tail + 255) / 256, 1024), 256, 0, st>>>(src + 16 * n16,
                                                                                           dst + 16 * n16, tail);
        note_launch();
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace

int stage_h2d(void* dst_dev, const void* src_host, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return LC_OK;
    if (bytes > kStageCap / 8)  // large enough to be worth a copy engine
        return cuda_status(cudaMemcpyAsync(dst_dev, src_host, bytes, cudaMemcpyHostToDevice, st));
    StageArena* a = nullptr;
    size_t off = 0;
    int rc = stage_reserve(bytes, st, &a, &off);
    if (rc) return rc;
    std::memcpy(a->h + off, src_host, bytes);
    return stage_copy(a->d + off, (uint8_t*)dst_dev, bytes, st);
}

int stage_d2h(const void* src_dev, size_t bytes, cudaStream_t st, const void** host_out) {
    StageArena* a = nullptr;
    size_t off = 0;
    int rc = stage_reserve(std::max<size_t>(bytes, 1), st, &a, &off);
    if (rc) return rc;
    *host_out = a->h + off;
    return bytes ? stage_copy((const uint8_t*)src_dev, a->d + off, bytes, st) : LC_OK;
}

int stage_sync(cudaStream_t st) {
    const int rc = cuda_status(cudaStreamSynchronize(st));
    StageArena* a = nullptr;
    if (!rc && stage_arena(&a) == LC_OK) a->off = 0;
    return rc;
}

static uint64_t pad16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

Layout make_layout(int kb, uint64_t C, uint64_t L, uint64_t W, uint64_t NL, bool list_mode) {
    Layout y;
    uint64_t off = 64;
    y.lkb = y.lcb = y.leps = y.llog = 0;
    if (list_mode) {
        y.lkb = off; off += pad16(8 * (NL + 1));
        y.lcb = off; off += pad16(8 * (NL + 1));
        y.leps = off; off += pad16(8 * NL);
        y.llog = off; off += pad16(NL);
    }
    y.ckb = off; off += pad16(8 * (C + 1));
    y.csb = off; off += pad16(8 * (C + 1));
    y.cwb = off; off += pad16(8 * (C + 1));
    y.icpt = off; off += pad16((uint64_t)kb * L);
    y.slope = off; off += pad16(8 * L);
    y.bitoff = off; off += pad16(4 * L);
    y.start = off; off += pad16(2 * L);
    y.width = off; off += pad16(L);
    y.payload = off; off += 8 * W;
    y.total = off;
    return y;
}

static void put(uint8_t* p, uint64_t v, int bytes) {
    for (int b = 0; b < bytes; ++b) p[b] = (uint8_t)(v >> (8 * b));
}
static uint64_t get(const uint8_t* p, int bytes) {
    uint64_t v = 0;
    for (int b = 0; b < bytes; ++b) v |= (uint64_t)p[b] << (8 * b);
    return v;
}

// Header, list directory and chunk_key_begin: everything in front of
// chunk_seg_begin, padding included.
static std::vector<uint8_t> build_prefix(const lc_column* col, const uint64_t* list_begin, const uint64_t* list_chunk_begin,
                                         const uint64_t* list_eps, const uint8_t* list_log2) {
    const Layout& y = col->lay;
    std::vector<uint8_t> b(y.csb, 0);
    memcpy(b.data(), "LCF1", 4);
    put(&b[4], 1, 2);
    put(&b[6], col->list_mode ? 1 : 0, 2);
    put(&b[8], col->key_bytes, 4);
    put(&b[12], col->chunk_log2, 4);
    put(&b[16], col->N, 8);
    put(&b[24], col->eps, 8);
    put(&b[32], col->C, 8);
    put(&b[40], col->L, 8);
    put(&b[48], col->W, 8);
    put(&b[56], col->NL, 8);
    if (col->list_mode) {
        for (uint64_t l = 0; l <= col->NL; ++l) {
            put(&b[y.lkb + 8 * l], list_begin[l], 8);
            put(&b[y.lcb + 8 * l], list_chunk_begin[l], 8);
        }
        for (uint64_t l = 0; l < col->NL; ++l) {
            put(&b[y.leps + 8 * l], list_eps[l], 8);
            b[y.llog + l] = list_log2[l];
        }
    }
    for (uint64_t c = 0; c <= col->C; ++c) put(&b[y.ckb + 8 * c], col->h_ckb[c], 8);
    return b;
}

// Keep up to an eighth of the device's memory (at least 8 GB) of freed pool
// memory mapped (once per device): a column's blob, directories and scratch
// are allocated and freed per call, several columns' worth can be in flight
// on concurrent streams, and re-mapping them after every synchronisation
// costs milliseconds.
constexpr uint64_t kPoolRetainMin = 8ull << 30;

static void retain_pool(int dev) {
    static std::once_flag once[64];
    if (dev < 0 || dev >= 64) return;
    std::call_once(once[dev], [dev] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
        size_t free_b = 0, total_b = 0;
        uint64_t want = kPoolRetainMin;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) want = std::max<uint64_t>(want, total_b / 8);
        uint64_t cur = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < want)
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &want);
    });
}

static lc_column* new_column() {
    lc_column* c = new (std::nothrow) lc_column;
    if (!c) return nullptr;
    memset((void*)c, 0, sizeof(*c));
    cudaGetDevice(&c->device);
    retain_pool(c->device);
    return c;
}

static unsigned bit_length(uint64_t x) {
    unsigned n = 0;
    while (x) { ++n; x >>= 1; }
    return n;
}

// Payload words if every residual of a chunk of n keys took the paper's
// ceil(log2(2 eps + 1)) bits (the largest any segment width can be).
static uint64_t bound_words(uint64_t n, uint64_t eps) {
    const uint64_t bits = (uint64_t)bit_length(2 * eps) * (n ? n - 1 : 0);
    const uint64_t w = (bits + 63) / 64;
    return w + (w & 1);
}

// Builds the empty-N or full column from a finished device blob.
static int finish_column(lc_column* col, cudaStream_t st, const uint64_t* lb, const uint64_t* lcb, const uint64_t* le,
                         const uint8_t* lg) {
    int rc;
    {
        HTime ht("finish_blob");
        std::vector<uint8_t> prefix = build_prefix(col, lb, lcb, le, lg);
        rc = finish_blob(col, prefix.data(), prefix.size(), st);
    }
    if (rc) return rc;
    HTime ht("derived");
    return build_derived(col, st);
}

static int alloc_empty_blob(lc_column* col, cudaStream_t st) {
    col->lay = make_layout((int)col->key_bytes, col->C, 0, 0, col->NL, col->list_mode != 0);
    col->blob_cap = col->lay.total;
    if (cudaMallocAsync((void**)&col->blob, col->lay.total, st) != cudaSuccess) {
        col->blob = nullptr;
        return LC_ERR_NOMEM;
    }
    return cuda_status(cudaMemsetAsync(col->blob, 0, col->lay.total, st));
}

}  // namespace lcx

using namespace lcx;

extern "C" {

int lc_version(void) { return 10000; }

uint64_t lc_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int lc_pool_usage(int reset, uint64_t* used_now, uint64_t* used_high) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&pool, dev);
    if (e == cudaSuccess && reset) {
        uint64_t zero = 0;  // resets the mark to the current use
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero);
    }
    uint64_t now = 0, high = 0;
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &now);
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high);
    if (e != cudaSuccess) return cuda_status(e);
    if (used_now) *used_now = now;
    if (used_high) *used_high = high;
    return LC_OK;
}

int lc_timing_enable(int on) {
    g_timing.store(on != 0);
    return LC_OK;
}

int lc_timing_read(lc_kernel_time* out, int max, int* got) {
    if (!got || (max > 0 && !out)) return LC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_timing_mu);
    for (TimedLaunch& t : g_timed) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.b) == cudaSuccess && cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            auto& e = g_totals[t.name];
            e.first += 1;
            e.second += ms;
        }
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    g_timed.clear();
    int n = 0;
    for (auto& kv : g_totals) {
        if (n >= max) break;
        memset(out[n].name, 0, sizeof(out[n].name));
        strncpy(out[n].name, kv.first.c_str(), sizeof(out[n].name) - 1);
        out[n].launches = kv.second.first;
        out[n].total_ms = kv.second.second;
        ++n;
    }
    g_totals.clear();
    *got = n;
    return LC_OK;
}

const char* lc_strerror(int s) {
    switch (s) {
        case LC_OK: return "ok";
        case LC_ERR_INVALID_ARG: return "invalid argument";
        case LC_ERR_UNSORTED: return "keys are not sorted";
        case LC_ERR_OUT_OF_RANGE: return "index out of range";
        case LC_ERR_NOMEM: return "out of memory";
        case LC_ERR_CORRUPT: return "corrupt blob";
        case LC_ERR_CUDA: return "CUDA error";
        case LC_ERR_TIMEOUT: return "timed out";
        case LC_ERR_BUSY: return "busy";
        case LC_ERR_UNSUPPORTED: return "unsupported for this column";
        case LC_ERR_INTERNAL: return "internal error";
        case LC_ERR_STALE: return "batch keys do not fit the planned layout";
        default: return "unknown status";
    }
}

void lc_free(lc_column* col) {
    if (!col) return;
    HTime ht("free");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != col->device) cudaSetDevice(col->device);
    cudaDeviceSynchronize();
    if (col->blob) cudaFree(col->blob);
    if (col->chunk_tile_begin) cudaFree(col->chunk_tile_begin);
    if (col->derived2) cudaFree(col->derived2);
    if (cur != col->device) cudaSetDevice(cur);
    delete[] col->h_ckb;
    delete[] col->h_ctb;
    delete col;
}

int lc_free_async(lc_column* col, void* stream) {
    if (!col) return LC_ERR_INVALID_ARG;
    HTime ht("free");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != col->device) cudaSetDevice(col->device);
    const cudaStream_t st = (cudaStream_t)stream;
    int rc = LC_OK;
    for (void* p : {(void*)col->blob, (void*)col->chunk_tile_begin, (void*)col->derived2})
        if (p && !rc) rc = cuda_status(cudaFreeAsync(p, st));
    if (cur != col->device) cudaSetDevice(cur);
    delete[] col->h_ckb;
    delete[] col->h_ctb;
    delete col;
    return rc;
}

static bool span_ok(uint32_t& span_log2) {
    if (span_log2 == 0) span_log2 = 6;
    return span_log2 >= 5 && span_log2 <= 7;
}

static int compress_column(const void* keys_dev, uint64_t n, int key_bytes, const lc_params* params, void* stream,
                           lc_column** out, bool jump);

int lc_compress(const void* keys_dev, uint64_t n, int key_bytes, const lc_params* params, void* stream,
                lc_column** out) {
    return compress_column(keys_dev, n, key_bytes, params, stream, out, false);
}

int lc_compress_jump(const void* keys_dev, uint64_t n, int key_bytes, const lc_params* params, void* stream,
                     lc_column** out) {
    return compress_column(keys_dev, n, key_bytes, params, stream, out, true);
}

static int compress_column(const void* keys_dev, uint64_t n, int key_bytes, const lc_params* params, void* stream,
                           lc_column** out, bool jump) {
    if (!out || (n && !keys_dev)) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    if (key_bytes != 4 && key_bytes != 8) return LC_ERR_INVALID_ARG;
    const uint64_t eps = params ? params->eps : 0;
    const uint32_t log2 = params ? params->chunk_log2 : 16;
    uint32_t span_log2 = params ? params->span_log2 : 0;
    if (eps > (1ull << 30) || log2 < 8 || log2 > 16 || !span_ok(span_log2)) return LC_ERR_INVALID_ARG;
    if (n > (1ull << 40)) return LC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    lc_column* col = new_column();
    if (!col) return LC_ERR_NOMEM;
    cudaGetDevice(&col->device);
    col->key_bytes = (uint32_t)key_bytes;
    col->chunk_log2 = log2;
    col->list_mode = 0;
    col->N = n;
    col->eps = eps;
    const uint64_t cs = 1ull << log2;
    col->C = (n + cs - 1) / cs;
    col->NL = 0;
    col->h_ckb = new (std::nothrow) uint64_t[col->C + 1];
    if (!col->h_ckb) { lc_free(col); return LC_ERR_NOMEM; }
    for (uint64_t c = 0; c <= col->C; ++c) col->h_ckb[c] = std::min(n, c * cs);
    int rc;
    if (n == 0) {
        rc = alloc_empty_blob(col, st);
    } else {
        std::vector<ChunkDesc> ch(col->C);
        uint64_t bound = 0;
        for (uint64_t c = 0; c < col->C; ++c) {
            ch[c].key_begin = c * cs;
            ch[c].bitword_begin = c * (cs / 32);
            ch[c].n = (uint32_t)(col->h_ckb[c + 1] - col->h_ckb[c]);
            ch[c].eps = (uint32_t)eps;
            ch[c].check_prev = c > 0;
            ch[c].pad = 0;
            bound += bound_words(ch[c].n, eps);
        }
        rc = compress_impl(keys_dev, key_bytes, ch.data(), col->C, col->C * (cs / 32), bound, st, col, jump,
                           span_log2);
    }
    if (!rc) rc = finish_column(col, st, nullptr, nullptr, nullptr, nullptr);
    if (rc) { lc_free(col); return rc; }
    *out = col;
    return LC_OK;
}

// The chunk table of a batch of lists (chunks restart at every list) and the
// list directory; fills col's list-mode fields.
struct BatchTable {
    std::vector<uint64_t> le, lcb;
    std::vector<uint8_t> lg;
    std::vector<ChunkDesc> ch;
    uint64_t bitwords = 0, bound = 0;
};

static int batch_table(const uint64_t* list_begin, uint64_t nlists, int key_bytes, const uint64_t* eps,
                       const uint8_t* chunk_log2, lc_column* col, BatchTable* bt) {
    col->key_bytes = (uint32_t)key_bytes;
    col->chunk_log2 = 0;
    col->list_mode = 1;
    col->N = list_begin[nlists];
    col->eps = 0;
    col->NL = nlists;
    bt->le.assign(nlists, 0);
    bt->lcb.assign(nlists + 1, 0);
    bt->lg.assign(nlists, 16);
    uint64_t C = 0;
    for (uint64_t l = 0; l < nlists; ++l) {
        bt->le[l] = eps ? eps[l] : 0;
        bt->lg[l] = chunk_log2 ? chunk_log2[l] : 16;
        const uint64_t cs = 1ull << bt->lg[l];
        bt->lcb[l] = C;
        C += (list_begin[l + 1] - list_begin[l] + cs - 1) / cs;
    }
    bt->lcb[nlists] = C;
    col->C = C;
    col->h_ckb = new (std::nothrow) uint64_t[C + 1];
    if (!col->h_ckb) return LC_ERR_NOMEM;
    bt->ch.resize(C);
    uint64_t c = 0;
    for (uint64_t l = 0; l < nlists; ++l) {
        const uint64_t cs = 1ull << bt->lg[l];
        for (uint64_t b = list_begin[l]; b < list_begin[l + 1]; b += cs, ++c) {
            const uint64_t e = std::min(b + cs, list_begin[l + 1]);
            col->h_ckb[c] = b;
            ChunkDesc& d = bt->ch[c];
            d.key_begin = b;
            d.bitword_begin = bt->bitwords;
            d.n = (uint32_t)(e - b);
            d.eps = (uint32_t)bt->le[l];
            d.check_prev = b > list_begin[l];
            d.pad = 0;
            bt->bitwords += (e - b + 31) / 32;
            bt->bound += bound_words(e - b, bt->le[l]);
        }
    }
    col->h_ckb[C] = col->N;
    return LC_OK;
}

static int check_batch_args(const void* ids_dev, const uint64_t* list_begin, uint64_t nlists, int key_bytes,
                            const uint64_t* eps, const uint8_t* chunk_log2) {
    if (!list_begin) return LC_ERR_INVALID_ARG;
    if (key_bytes != 4 && key_bytes != 8) return LC_ERR_INVALID_ARG;
    if (list_begin[0] != 0) return LC_ERR_INVALID_ARG;
    for (uint64_t l = 0; l < nlists; ++l) {
        if (list_begin[l + 1] < list_begin[l]) return LC_ERR_INVALID_ARG;
        if (eps && eps[l] > (1ull << 30)) return LC_ERR_INVALID_ARG;
        if (chunk_log2 && (chunk_log2[l] < 8 || chunk_log2[l] > 16)) return LC_ERR_INVALID_ARG;
    }
    const uint64_t n = list_begin[nlists];
    if (n && !ids_dev) return LC_ERR_INVALID_ARG;
    if (n > (1ull << 40)) return LC_ERR_INVALID_ARG;
    return LC_OK;
}

int lc_compress_batch(const void* ids_dev, const uint64_t* list_begin, uint64_t nlists, int key_bytes,
                      const uint64_t* eps, const uint8_t* chunk_log2, uint32_t span_log2, void* stream,
                      lc_column** out) {
    if (!out) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!span_ok(span_log2)) return LC_ERR_INVALID_ARG;
    int rc = check_batch_args(ids_dev, list_begin, nlists, key_bytes, eps, chunk_log2);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    lc_column* col = new_column();
    if (!col) return LC_ERR_NOMEM;
    BatchTable bt;
    rc = batch_table(list_begin, nlists, key_bytes, eps, chunk_log2, col, &bt);
    if (!rc) rc = col->C == 0 ? alloc_empty_blob(col, st)
                              : compress_impl(ids_dev, key_bytes, bt.ch.data(), col->C, bt.bitwords, bt.bound, st, col,
                                              false, span_log2);
    if (!rc) rc = finish_column(col, st, list_begin, bt.lcb.data(), bt.le.data(), bt.lg.data());
    if (rc) { lc_free(col); return rc; }
    *out = col;
    return LC_OK;
}

struct lc_batch {
    lc_column* col;
    lcx::BatchGraph* graph;
};

int lc_batch_create(const void* ids_dev, const uint64_t* list_begin, uint64_t nlists, int key_bytes,
                    const uint64_t* eps, const uint8_t* chunk_log2, uint32_t span_log2, void* out_dev, void* stream,
                    lc_batch** out) {
    if (!out) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!span_ok(span_log2)) return LC_ERR_INVALID_ARG;
    int rc = check_batch_args(ids_dev, list_begin, nlists, key_bytes, eps, chunk_log2);
    if (rc) return rc;
    if (list_begin[nlists] == 0 || !out_dev || ((uintptr_t)out_dev % key_bytes)) return LC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    lc_column* col = new_column();
    if (!col) return LC_ERR_NOMEM;
    BatchTable bt;
    rc = batch_table(list_begin, nlists, key_bytes, eps, chunk_log2, col, &bt);
    if (!rc) rc = compress_impl(ids_dev, key_bytes, bt.ch.data(), col->C, bt.bitwords, bt.bound, st, col, false,
                                span_log2);
    if (!rc) rc = finish_column(col, st, list_begin, bt.lcb.data(), bt.le.data(), bt.lg.data());
    BatchGraph* g = nullptr;
    if (!rc)
        rc = batch_graph_build(ids_dev, key_bytes, bt.ch.data(), col->C, bt.bitwords, span_log2, col, out_dev, st, &g);
    lc_batch* b = nullptr;
    if (!rc) {
        b = new (std::nothrow) lc_batch{col, g};
        if (!b) rc = LC_ERR_NOMEM;
    }
    if (rc) {
        batch_graph_free(g);
        lc_free(col);
        return rc;
    }
    *out = b;
    return LC_OK;
}

int lc_batch_launch(lc_batch* b, void* stream) {
    if (!b) return LC_ERR_INVALID_ARG;
    return batch_graph_launch(b->graph, (cudaStream_t)stream);
}

const lc_column* lc_batch_column(const lc_batch* b) { return b ? b->col : nullptr; }

void lc_batch_free(lc_batch* b) {
    if (!b) return;
    batch_graph_free(b->graph);
    lc_free(b->col);
    delete b;
}

// Output keys are stored whole: the buffer must be aligned to the key width.
static bool misaligned(const lc_column* col, const void* out) {
    return ((uintptr_t)out % col->key_bytes) != 0;
}

int lc_decode(const lc_column* col, uint64_t begin, uint64_t count, void* out_dev, void* stream) {
    if (!col || (count && !out_dev) || misaligned(col, out_dev)) return LC_ERR_INVALID_ARG;
    if (begin > col->N || count > col->N - begin) return LC_ERR_OUT_OF_RANGE;
    return decode_range(col, begin, count, out_dev, (cudaStream_t)stream);
}

int lc_decode_ranges(const lc_column* col, const uint64_t* begin_dev, const uint64_t* count_dev,
                     const uint64_t* out_off_dev, uint64_t m, void* out_dev, uint64_t out_cap, void* stream) {
    if (!col || (m && (!begin_dev || !count_dev || !out_off_dev || !out_dev))) return LC_ERR_INVALID_ARG;
    if (misaligned(col, out_dev)) return LC_ERR_INVALID_ARG;
    if (col->N == 0) return LC_OK;
    return decode_ranges(col, begin_dev, count_dev, out_off_dev, m, out_dev, out_cap, (cudaStream_t)stream);
}

int lc_decode_ranges_noalloc(const lc_column* col, const uint64_t* begin_dev, const uint64_t* count_dev,
                             const uint64_t* out_off_dev, uint64_t m, void* out_dev, uint64_t out_cap,
                             void* stream) {
    if (!col || (m && (!begin_dev || !count_dev || !out_off_dev || !out_dev))) return LC_ERR_INVALID_ARG;
    if (m > LC_NOALLOC_MAX_RANGES || misaligned(col, out_dev)) return LC_ERR_INVALID_ARG;
    if (col->N == 0) return LC_OK;
    return decode_ranges_noalloc(col, begin_dev, count_dev, out_off_dev, m, out_dev, out_cap, (cudaStream_t)stream);
}

int lc_decode_batch(const lc_column* col, void* out_dev, void* stream) {
    if (!col) return LC_ERR_INVALID_ARG;
    return lc_decode(col, 0, col->N, out_dev, stream);
}

struct lc_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

int lc_graph_decode(const lc_column* col, uint64_t begin, uint64_t count, void* out_dev, void* stream, lc_graph** out) {
    if (!col || !out || (count && !out_dev)) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    if (begin > col->N || count > col->N - begin) return LC_ERR_OUT_OF_RANGE;
    cudaStream_t st = (cudaStream_t)stream, own = nullptr;
    if (!st) {
        if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess) return LC_ERR_CUDA;
        st = own;
    }
    // one eager run sets the kernel attributes outside the capture
    int rc = decode_range(col, begin, count, out_dev, st);
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    lc_graph* g = nullptr;
    if (!rc) {
        g = new (std::nothrow) lc_graph{nullptr, nullptr};
        if (!g) rc = LC_ERR_NOMEM;
    }
    if (!rc) rc = cuda_status(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    if (!rc) {
        const int rk = decode_range(col, begin, count, out_dev, st);
        const int re = cuda_status(cudaStreamEndCapture(st, &g->graph));
        rc = rk ? rk : re;
    }
    if (!rc) rc = cuda_status(cudaGraphInstantiate(&g->exec, g->graph, 0));
    if (own) cudaStreamDestroy(own);
    if (rc) {
        if (g) {
            if (g->graph) cudaGraphDestroy(g->graph);
            delete g;
        }
        return rc;
    }
    *out = g;
    return LC_OK;
}

int lc_graph_launch(lc_graph* g, void* stream) {
    if (!g) return LC_ERR_INVALID_ARG;
    return cuda_status(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
}

void lc_graph_free(lc_graph* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

int lc_access(const lc_column* col, const uint64_t* idx_dev, uint64_t m, void* out_dev, void* stream) {
    if (!col || (m && (!idx_dev || !out_dev))) return LC_ERR_INVALID_ARG;
    if (col->N == 0) {
        if (m) {
            cudaMemsetAsync(out_dev, 0, m * col->key_bytes, (cudaStream_t)stream);
            uint32_t bit = kStOutOfRange;
            cudaMemcpyAsync(col->status, &bit, 4, cudaMemcpyHostToDevice, (cudaStream_t)stream);
            cudaStreamSynchronize((cudaStream_t)stream);
        }
        return LC_OK;
    }
    return access(col, idx_dev, m, out_dev, (cudaStream_t)stream);
}

int lc_lower_bound(const lc_column* col, const void* v_dev, uint64_t m, uint64_t* out_dev, void* stream) {
    if (!col || (m && (!v_dev || !out_dev))) return LC_ERR_INVALID_ARG;
    if (col->list_mode) return LC_ERR_UNSUPPORTED;
    return lower_bound(col, v_dev, m, out_dev, (cudaStream_t)stream);
}

int lc_set_query_plan(int plan) { return set_query_plan(plan); }

// ------------------------------------------------------------------ host-buffer entry points
//
// The same calls with inputs and outputs in host memory: the library copies
// them to and from device buffers it takes from the stream-ordered pool and
// releases in stream order.  With page-locked host memory every copy is
// asynchronous on `stream`, so that calls on several streams overlap their
// copies with one another's kernels.

namespace {
struct DevBuf {
    void* p = nullptr;
    cudaStream_t st;
    explicit DevBuf(cudaStream_t s) : st(s) {}
    int alloc(size_t bytes) {
        if (!bytes) return LC_OK;
        return cudaMallocAsync(&p, bytes, st) == cudaSuccess ? LC_OK : (p = nullptr, LC_ERR_NOMEM);
    }
    ~DevBuf() {
        if (p) cudaFreeAsync(p, st);
    }
};
int h2d(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    return bytes ? cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st)) : LC_OK;
}
int d2h(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    return bytes ? cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st)) : LC_OK;
}
}  // namespace

int lc_compress_host(const void* keys_host, uint64_t n, int key_bytes, const lc_params* params, void* stream,
                     lc_column** out) {
    if (!out || (n && !keys_host) || (key_bytes != 4 && key_bytes != 8)) return LC_ERR_INVALID_ARG;
    if (n > (1ull << 40)) return LC_ERR_INVALID_ARG;
    const cudaStream_t st = (cudaStream_t)stream;
    DevBuf k(st);
    int rc = k.alloc(n * (uint64_t)key_bytes);
    if (!rc) rc = h2d(k.p, keys_host, n * (uint64_t)key_bytes, st);
    if (rc) return rc;
    return compress_column(k.p, n, key_bytes, params, stream, out, false);
}

int lc_decode_host(const lc_column* col, uint64_t begin, uint64_t count, void* out_host, void* stream) {
    if (!col || (count && !out_host)) return LC_ERR_INVALID_ARG;
    if (begin > col->N || count > col->N - begin) return LC_ERR_OUT_OF_RANGE;
    const cudaStream_t st = (cudaStream_t)stream;
    DevBuf o(st);
    int rc = o.alloc(count * col->key_bytes);
    if (!rc && count) rc = decode_range(col, begin, count, o.p, st);
    if (!rc) rc = d2h(out_host, o.p, count * col->key_bytes, st);
    return rc;
}

int lc_decode_ranges_host(const lc_column* col, const uint64_t* begin_host, const uint64_t* count_host,
                          const uint64_t* out_off_host, uint64_t m, void* out_host, uint64_t out_cap, void* stream) {
    if (!col || (m && (!begin_host || !count_host || !out_off_host || (out_cap && !out_host))))
        return LC_ERR_INVALID_ARG;
    if (col->N == 0 || m == 0) return LC_OK;
    const cudaStream_t st = (cudaStream_t)stream;
    DevBuf in(st), o(st);
    int rc = in.alloc(24 * m);
    if (!rc) rc = o.alloc(out_cap * col->key_bytes);
    uint64_t* b = (uint64_t*)in.p;
    if (!rc) rc = h2d(b, begin_host, 8 * m, st);
    if (!rc) rc = h2d(b + m, count_host, 8 * m, st);
    if (!rc) rc = h2d(b + 2 * m, out_off_host, 8 * m, st);
    if (!rc) rc = decode_ranges(col, b, b + m, b + 2 * m, m, o.p, out_cap, st);
    if (!rc) rc = d2h(out_host, o.p, out_cap * col->key_bytes, st);
    return rc;
}

int lc_access_host(const lc_column* col, const uint64_t* idx_host, uint64_t m, void* out_host, void* stream) {
    if (!col || (m && (!idx_host || !out_host))) return LC_ERR_INVALID_ARG;
    if (m == 0) return LC_OK;
    const cudaStream_t st = (cudaStream_t)stream;
    DevBuf in(st), o(st);
    int rc = in.alloc(8 * m);
    if (!rc) rc = o.alloc(m * col->key_bytes);
    if (!rc) rc = h2d(in.p, idx_host, 8 * m, st);
    if (!rc) rc = lc_access(col, (const uint64_t*)in.p, m, o.p, stream);
    if (!rc) rc = d2h(out_host, o.p, m * col->key_bytes, st);
    return rc;
}

int lc_lower_bound_host(const lc_column* col, const void* v_host, uint64_t m, uint64_t* out_host, void* stream) {
    if (!col || (m && (!v_host || !out_host))) return LC_ERR_INVALID_ARG;
    if (col->list_mode) return LC_ERR_UNSUPPORTED;
    if (m == 0) return LC_OK;
    const cudaStream_t st = (cudaStream_t)stream;
    DevBuf in(st), o(st);
    int rc = in.alloc(m * col->key_bytes);
    if (!rc) rc = o.alloc(8 * m);
    if (!rc) rc = h2d(in.p, v_host, m * col->key_bytes, st);
    if (!rc) rc = lower_bound(col, in.p, m, (uint64_t*)o.p, st);
    if (!rc) rc = d2h(out_host, o.p, 8 * m, st);
    return rc;
}

int lc_quantile(const lc_column* col, const uint64_t* k_dev, uint64_t m, uint64_t q, int exact, void* out_dev,
                void* stream) {
    if (!col || q == 0 || (m && (!k_dev || !out_dev))) return LC_ERR_INVALID_ARG;
    if (col->list_mode) return LC_ERR_UNSUPPORTED;
    if (col->N == 0) return m ? LC_ERR_OUT_OF_RANGE : LC_OK;
    return quantile(col, k_dev, m, q, exact ? 1 : 0, out_dev, (cudaStream_t)stream);
}

int lc_decode_approx(const lc_column* col, uint64_t begin, uint64_t count, void* out_dev, void* stream) {
    if (!col || (count && !out_dev)) return LC_ERR_INVALID_ARG;
    if (begin > col->N || count > col->N - begin) return LC_ERR_OUT_OF_RANGE;
    return decode_approx(col, begin, count, out_dev, (cudaStream_t)stream);
}

int lc_intersect(const lc_column* a, int64_t la, const lc_column* b, int64_t lb, void* out_dev, uint64_t cap,
                 uint64_t* count, void* stream) {
    if (!a || !b || !count) return LC_ERR_INVALID_ARG;
    return set_op(true, a, la, b, lb, out_dev, cap, count, (cudaStream_t)stream);
}

int lc_union(const lc_column* a, int64_t la, const lc_column* b, int64_t lb, void* out_dev, uint64_t cap,
             uint64_t* count, void* stream) {
    if (!a || !b || !count) return LC_ERR_INVALID_ARG;
    return set_op(false, a, la, b, lb, out_dev, cap, count, (cudaStream_t)stream);
}

int lc_chunk_bytes(const lc_column* col, uint64_t* out_host, uint64_t cap) {
    if (!col || (col->C && !out_host)) return LC_ERR_INVALID_ARG;
    if (cap < col->C) return LC_ERR_INVALID_ARG;
    if (col->C == 0) return LC_OK;
    std::vector<uint64_t> csb(col->C + 1), cwb(col->C + 1);
    int rc = cuda_status(cudaMemcpy(csb.data(), col->blob + col->lay.csb, 8 * (col->C + 1), cudaMemcpyDeviceToHost));
    if (!rc) rc = cuda_status(cudaMemcpy(cwb.data(), col->blob + col->lay.cwb, 8 * (col->C + 1), cudaMemcpyDeviceToHost));
    if (rc) return rc;
    const uint64_t seg_bytes = (uint64_t)col->key_bytes + 8 + 4 + 2 + 1;  // icpt, slope, bitoff, start, width
    for (uint64_t c = 0; c < col->C; ++c)
        out_host[c] = (csb[c + 1] - csb[c]) * seg_bytes + 8 * (cwb[c + 1] - cwb[c]) + 24;  // + 3 directory entries
    return LC_OK;
}

int lc_access1(const lc_column* col, uint64_t i, uint64_t* key) {
    if (!col || !key) return LC_ERR_INVALID_ARG;
    if (i >= col->N) return LC_ERR_OUT_OF_RANGE;
    uint64_t* buf = nullptr;
    if (cudaMalloc((void**)&buf, 16) != cudaSuccess) return LC_ERR_NOMEM;
    int rc = cuda_status(cudaMemcpy(buf, &i, 8, cudaMemcpyHostToDevice));
    if (!rc) rc = access(col, buf, 1, buf + 1, nullptr);
    uint64_t v = 0;
    if (!rc) rc = cuda_status(cudaMemcpy(&v, buf + 1, 8, cudaMemcpyDeviceToHost));
    cudaFree(buf);
    if (!rc) *key = col->key_bytes == 4 ? (uint32_t)v : v;
    return rc;
}

int lc_lower_bound1(const lc_column* col, uint64_t x, uint64_t* pos) {
    if (!col || !pos) return LC_ERR_INVALID_ARG;
    if (col->list_mode) return LC_ERR_UNSUPPORTED;
    if (col->key_bytes == 4 && x > 0xFFFFFFFFull) {
        *pos = col->N;
        return LC_OK;
    }
    uint64_t* buf = nullptr;
    if (cudaMalloc((void**)&buf, 16) != cudaSuccess) return LC_ERR_NOMEM;
    int rc = cuda_status(cudaMemcpy(buf, &x, col->key_bytes, cudaMemcpyHostToDevice));
    if (!rc) rc = lower_bound(col, buf, 1, buf + 1, nullptr);
    if (!rc) rc = cuda_status(cudaMemcpy(pos, buf + 1, 8, cudaMemcpyDeviceToHost));
    cudaFree(buf);
    return rc;
}

double lc_ratio(const lc_column* col) {
    if (!col) return -1.0;
    if (col->N == 0) return 0.0;
    return (double)col->lay.total / ((double)col->N * (double)col->key_bytes);
}

int lc_size(const lc_column* col, uint64_t* bytes) {
    if (!col || !bytes) return LC_ERR_INVALID_ARG;
    *bytes = col->lay.total;
    return LC_OK;
}

int lc_info(const lc_column* col, lc_info_t* info) {
    if (!col || !info) return LC_ERR_INVALID_ARG;
    info->n = col->N;
    info->chunks = col->C;
    info->segments = col->L;
    info->words = col->W;
    info->lists = col->NL;
    info->bytes = col->lay.total;
    info->eps = col->eps;
    info->key_bytes = col->key_bytes;
    info->chunk_log2 = col->chunk_log2;
    return LC_OK;
}

int lc_serialize(const lc_column* col, void* host, uint64_t cap, uint64_t* len) {
    if (!col || !len) return LC_ERR_INVALID_ARG;
    *len = col->lay.total;
    if (!host || cap < col->lay.total) return LC_ERR_INVALID_ARG;
    return cuda_status(cudaMemcpy(host, col->blob, col->lay.total, cudaMemcpyDeviceToHost));
}

// Structural validation of an LCF1 blob on the host: every fact of the format
// is checked before anything is uploaded.
static int validate_blob(const uint8_t* b, uint64_t len, lc_column* col) {
    if (len < 64 || memcmp(b, "LCF1", 4) != 0 || get(b + 4, 2) != 1) return LC_ERR_CORRUPT;
    const uint64_t flags = get(b + 6, 2);
    if (flags > 1) return LC_ERR_CORRUPT;
    const bool lm = flags == 1;
    const uint64_t kb = get(b + 8, 4), log2 = get(b + 12, 4), N = get(b + 16, 8), eps = get(b + 24, 8);
    const uint64_t C = get(b + 32, 8), L = get(b + 40, 8), W = get(b + 48, 8), NL = get(b + 56, 8);
    if (kb != 4 && kb != 8) return LC_ERR_CORRUPT;
    const uint64_t lim = 1ull << 40;
    if (N > lim || C > lim || L > lim || W > lim || NL > lim) return LC_ERR_CORRUPT;
    if (lm ? (log2 != 0 || eps != 0) : (log2 < 8 || log2 > 16 || eps > (1ull << 30) || NL != 0)) return LC_ERR_CORRUPT;
    const Layout y = make_layout((int)kb, C, L, W, NL, lm);
    if (y.total != len) return LC_ERR_CORRUPT;
    // padding bytes between arrays are zero
    struct Ar { uint64_t off, bytes; };
    std::vector<Ar> arrs;
    if (lm) arrs.insert(arrs.end(), {{y.lkb, 8 * (NL + 1)}, {y.lcb, 8 * (NL + 1)}, {y.leps, 8 * NL}, {y.llog, NL}});
    arrs.insert(arrs.end(), {{y.ckb, 8 * (C + 1)}, {y.csb, 8 * (C + 1)}, {y.cwb, 8 * (C + 1)}, {y.icpt, kb * L},
                             {y.slope, 8 * L}, {y.bitoff, 4 * L}, {y.start, 2 * L}, {y.width, L}});
    for (const Ar& a : arrs)
        for (uint64_t i = a.off + a.bytes; i < pad16(a.off + a.bytes); ++i)
            if (b[i]) return LC_ERR_CORRUPT;
    auto U = [&](uint64_t off, uint64_t i) { return get(b + off + 8 * i, 8); };
    if (U(y.ckb, 0) || U(y.csb, 0) || U(y.cwb, 0)) return LC_ERR_CORRUPT;
    if (U(y.ckb, C) != N || U(y.csb, C) != L || U(y.cwb, C) != W) return LC_ERR_CORRUPT;
    for (uint64_t c = 0; c < C; ++c) {
        const uint64_t k0 = U(y.ckb, c), k1 = U(y.ckb, c + 1), s0 = U(y.csb, c), s1 = U(y.csb, c + 1);
        const uint64_t w0 = U(y.cwb, c), w1 = U(y.cwb, c + 1);
        if (k1 <= k0 || k1 - k0 > kMaxChunk || s1 <= s0 || s1 > L || w1 < w0 || ((w1 - w0) & 1)) return LC_ERR_CORRUPT;
        const uint64_t nc = k1 - k0;
        uint64_t bits = 0;
        for (uint64_t j = s0; j < s1; ++j) {
            const uint64_t st = get(b + y.start + 2 * j, 2);
            const uint64_t en = j + 1 < s1 ? get(b + y.start + 2 * (j + 1), 2) : nc;
            if ((j == s0 && st != 0) || en <= st || en > nc) return LC_ERR_CORRUPT;
            const uint64_t w = b[y.width + j];
            if (w > 32 || get(b + y.bitoff + 4 * j, 4) != bits) return LC_ERR_CORRUPT;
            bits += w * (en - st - 1);
        }
        uint64_t words = (bits + 63) / 64;
        words += words & 1;
        if (w1 - w0 != words) return LC_ERR_CORRUPT;
        for (uint64_t p = bits; p < 64 * words; ++p) {  // unused payload bits are zero
            const uint64_t gp = 64 * w0 + p;
            if ((b[y.payload + (gp >> 3)] >> (gp & 7)) & 1) return LC_ERR_CORRUPT;
        }
    }
    if (!lm) {
        const uint64_t cs = 1ull << log2;
        if (C != (N + cs - 1) / cs) return LC_ERR_CORRUPT;
        for (uint64_t c = 0; c < C; ++c)
            if (U(y.ckb, c) != c * cs) return LC_ERR_CORRUPT;
    } else {
        if (U(y.lkb, 0) || U(y.lcb, 0) || U(y.lkb, NL) != N || U(y.lcb, NL) != C) return LC_ERR_CORRUPT;
        for (uint64_t l = 0; l < NL; ++l) {
            const uint64_t a = U(y.lkb, l), e = U(y.lkb, l + 1), ca = U(y.lcb, l), cb = U(y.lcb, l + 1);
            const uint64_t lg = b[y.llog + l];
            if (e < a || cb < ca || lg < 8 || lg > 16 || U(y.leps, l) > (1ull << 30)) return LC_ERR_CORRUPT;
            const uint64_t cs = 1ull << lg;
            if (cb - ca != (e - a + cs - 1) / cs) return LC_ERR_CORRUPT;
            for (uint64_t c = ca; c < cb; ++c)
                if (U(y.ckb, c) != a + (c - ca) * cs) return LC_ERR_CORRUPT;
        }
    }
    col->key_bytes = (uint32_t)kb;
    col->chunk_log2 = (uint32_t)log2;
    col->list_mode = lm;
    col->N = N;
    col->eps = eps;
    col->C = C;
    col->L = L;
    col->W = W;
    col->NL = NL;
    col->lay = y;
    col->h_ckb = new (std::nothrow) uint64_t[C + 1];
    if (!col->h_ckb) return LC_ERR_NOMEM;
    for (uint64_t c = 0; c <= C; ++c) col->h_ckb[c] = U(y.ckb, c);
    return LC_OK;
}

int lc_deserialize(const void* host, uint64_t len, void* stream, lc_column** out) {
    if (!host || !out) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    lc_column* col = new_column();
    if (!col) return LC_ERR_NOMEM;
    cudaGetDevice(&col->device);
    int rc = validate_blob((const uint8_t*)host, len, col);
    if (rc) { lc_free(col); return rc; }
    cudaStream_t st = (cudaStream_t)stream;
    col->blob_cap = len;
    if (cudaMallocAsync((void**)&col->blob, len, st) != cudaSuccess) {  // stream-ordered, like lc_compress's
        col->blob = nullptr;
        lc_free(col);
        return LC_ERR_NOMEM;
    }
    rc = cuda_status(cudaMemcpyAsync(col->blob, host, len, cudaMemcpyHostToDevice, st));
    if (!rc) rc = build_derived(col, st);
    if (rc) { lc_free(col); return rc; }
    *out = col;
    return LC_OK;
}

int lc_selftest_wait(uint32_t polls, void* stream) {
    if (polls == 0 || polls > (1u << 20)) return LC_ERR_INVALID_ARG;
    return wait_selftest(polls, (cudaStream_t)stream);
}

int lc_status(const lc_column* col, void* stream) {
    if (!col) return LC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t s = 0;
    int rc = cuda_status(cudaStreamSynchronize(st));
    if (rc) return rc;
    rc = cuda_status(cudaMemcpy(&s, col->status, 4, cudaMemcpyDeviceToHost));
    if (rc) return rc;
    if (s) cudaMemset(col->status, 0, 4);
    if (s & kStOutOfRange) return LC_ERR_OUT_OF_RANGE;
    if (s & kStUnsorted) return LC_ERR_UNSORTED;
    if (s & kStTimeout) return LC_ERR_TIMEOUT;
    if (s & kStPlan) return LC_ERR_STALE;
    if (s) return LC_ERR_INTERNAL;
    return LC_OK;
}

}  // extern "C"
