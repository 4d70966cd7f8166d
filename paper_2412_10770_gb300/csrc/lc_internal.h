// lc_internal.h -- internal structures shared by the translation units of the
// GB300 learned-compression library (not part of the public C ABI).
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/lc.h"

namespace lcx {

// Keys decoded by one CTA of the decode kernel.  Tiles never cross a chunk.
constexpr int kTileLog = 11;
constexpr uint32_t kTile = 1u << kTileLog;
// A chunk holds at most 2^16 keys.
constexpr uint32_t kMaxChunk = 1u << 16;

// Device status bits (OR-ed by kernels, read by lc_status / lc_compress).
enum : uint32_t {
    kStUnsorted = 1u,
    kStOutOfRange = 2u,
    kStInternal = 4u,
    kStTimeout = 8u,
    kStPlan = 16u,  // a batch graph replay does not fit its plan
};

// One chunk of the fit: keys [key_begin, key_begin + n) of the input, error
// bound eps, and where its anchor bits live in the bitmap.
struct ChunkDesc {
    uint64_t key_begin;
    uint64_t bitword_begin;  // first 32-bit word of this chunk's anchor bitmap
    uint32_t n;
    uint32_t eps;
    uint32_t check_prev;  // 1: K[key_begin - 1] <= K[key_begin] must hold (same list)
    uint32_t pad;
};

// A speculation window of the fit: keys [off, off + 8192) of chunk `chunk`.
struct WinDesc {
    uint32_t chunk;
    uint32_t off;
};

// One request of a serving batch, as the device sees it.
struct SrvReq {
    uint64_t begin;       // LC_OP_DECODE: first key
    uint64_t count;       // queries (access, lower_bound) or keys (decode)
    uint64_t qoff;        // access / lower_bound: first query of the request in the batch
    uint64_t first_tile;  // decode: first tile
    uint64_t out;         // decode: device address of the request's keys
    uint32_t col;
    uint32_t op;
};

// A decode tile: keys [key_begin, key_begin + n) of chunk `chunk`; its first
// and last keys lie in segments seg_lo and seg_hi (global segment indices);
// their residuals lie in the 32-bit payload words [pw0, pw0 + pwn) (pw0 and
// pwn multiples of 4, so that the window is a 16-byte aligned run).
struct TileDesc {
    uint64_t key_begin;
    uint64_t seg_lo;
    uint64_t seg_hi;
    uint64_t pw0;
    uint32_t chunk;
    uint32_t n;
    uint32_t pwn;
    uint32_t pad;
};
static_assert(sizeof(TileDesc) == 48, "TileDesc layout");

// Derived (not serialized) directories of a column, built on the device when a
// column is created.  They put everything one random query needs into few
// sectors.
//
// SegRec: one segment's model in 32 bytes (one sector): intercept K[s_j],
// Q32 slope, the global index of its anchor with the width in the top byte,
// and the global payload bit of its residual t = 1 with the segment's key
// count n_j - 1 in the top 16 bits.
struct SegRec {
    uint64_t icpt;
    int64_t slope;
    uint64_t kstart_w;  // anchor key index (low 56 bits) | width << 56
    uint64_t bit1_n;    // payload bit of residual 1 (low 48 bits) | (n_j - 1) << 48
};
static_assert(sizeof(SegRec) == 32, "records are read with one 32-byte load");
constexpr uint64_t kBitMask = (1ull << 48) - 1;
// RankWord: anchor bits of keys [64q, 64q + 64) and the number of anchors
// before key 64q, so that the segment of key i is
// before + popcount(bits & mask(i)) - 1.
struct RankWord {
    uint64_t bits;
    uint64_t before;
};
// The radix table used by lower_bound: the value range [kmin, kmax] of the
// intercepts is cut into B = 2^b equal buckets of 2^rdx_shift values, and
// rdx[q] = the number of segments whose intercept is < kmin + q 2^rdx_shift
// (q = 0..B).  A value x in bucket q has its last segment with intercept < x
// among rdx[q] - 1 .. rdx[q+1] - 1.
constexpr uint32_t kRdxMaxLog = 22;

// Byte offsets of every array inside an LCF1 blob.
struct Layout {
    uint64_t lkb, lcb, leps, llog;          // list mode only
    uint64_t ckb, csb, cwb;                 // chunk directory
    uint64_t icpt, slope, bitoff, start, width, payload;
    uint64_t total;                          // exact blob length
};

Layout make_layout(int kb, uint64_t C, uint64_t L, uint64_t W, uint64_t NL, bool list_mode);

// Read-only device view of a column, passed to kernels by value.
struct ColView {
    const uint64_t* ckb;  // chunk_key_begin [C+1]
    const uint64_t* csb;  // chunk_seg_begin [C+1]
    const uint64_t* cwb;  // chunk_word_begin [C+1]
    const void* icpt;     // [L] key_bytes each
    const int64_t* slope;
    const uint32_t* bitoff;
    const uint16_t* start;
    const uint8_t* width;
    const uint32_t* pay32;  // payload as 32-bit little-endian words [2W]
    const TileDesc* tiles;
    const uint64_t* chunk_tile_begin;  // [C+1]
    const SegRec* recs;                // [L]
    const RankWord* rank;              // [ceil(N / 64)]
    const uint64_t* rdx;               // radix table over the intercepts [B + 1]
    const void* ioff;                  // [L] intercept - its bucket's first value, ioff_bytes each
    uint64_t kmin, kmax;               // first and last key
    uint32_t rdx_shift;                // bucket width 2^rdx_shift
    uint32_t ioff_bytes;               // 2 or 4; 0: no offsets (buckets wider than 2^32), use icpt
    uint32_t max_tile_segs;            // most segments meeting one decode tile
    uint32_t key_bytes;
    uint32_t* status;
    const uint32_t* gate;  // batch graph replays: the kernels that read the column do nothing while *gate == 0
    uint64_t N, C, L, W, ntiles;
    uint32_t chunk_log2;  // 0 in list mode
    uint32_t list_mode;
};

}  // namespace lcx

// The opaque column of the public ABI.
struct lc_column {
    int device;
    uint32_t key_bytes, chunk_log2, list_mode;
    uint64_t N, eps, C, L, W, NL;
    lcx::Layout lay;
    uint8_t* blob;            // device, exact LCF1 bytes (allocation may be larger)
    uint64_t blob_cap;
    lcx::TileDesc* tiles;     // device, derived
    uint64_t ntiles;
    uint64_t* chunk_tile_begin;  // device [C+1], derived
    uint8_t* derived2;           // device: SegRec, RankWord and the radix table
    uint32_t* status;            // device status word
    uint64_t* h_ckb;             // host copy of chunk_key_begin [C+1]
    uint64_t* h_ctb;             // host copy of chunk_tile_begin [C+1]
    lcx::ColView view;
};

namespace lcx {

// Compression pipeline (lc_compress.cu).  chunks_h: C chunk descriptors (host).
// Allocates col->blob and fills everything but the prefix (header, list
// directory, chunk_key_begin) and the padding bytes; sets col->L, col->W and
// col->lay.  Synchronizes `st`.
// span_log2: keys per speculating thread of the fit, 2^5, 2^6 or 2^7 (the bytes do not depend on it).
int compress_impl(const void* keys_dev, int kb, const ChunkDesc* chunks_h, uint64_t C, uint64_t bitwords,
                  uint64_t payload_bound_words, cudaStream_t st, lc_column* col, bool jump = false,
                  uint32_t span_log2 = 6);
// The batching graph (lc_batch_*): records a replay of the compress that
// made `col` (same chunk table) and a decode of every key into out_dev.
struct BatchGraph;
int batch_graph_build(const void* keys_dev, int kb, const ChunkDesc* chunks_h, uint64_t C, uint64_t bitwords,
                      uint32_t span_log2, lc_column* col, void* out_dev, cudaStream_t st, BatchGraph** out);
int batch_graph_launch(BatchGraph* g, cudaStream_t st);
void batch_graph_free(BatchGraph* g);
// Enqueue only (no host synchronisation): the list-mode derived directories
// (tile directory, segment records, rank words) and a decode of every key,
// all gated by *gate.  tmp: derived_replay_tmp_bytes(col) bytes of device scratch.
size_t derived_replay_tmp_bytes(const lc_column* col);
int derived_replay(lc_column* col, const uint32_t* gate, void* tmp, size_t tmp_bytes, void* out, cudaStream_t st);
// Upload the host-built prefix of the blob and zero its padding bytes.
int finish_blob(lc_column* col, const uint8_t* prefix_h, uint64_t prefix_len, cudaStream_t st);

// Derived directories and the kernel view (lc_query.cu).  build_derived
// takes col->derived2 as it finds it when it is set (derived2_layout(N, L,
// list_mode).bytes of device memory), else allocates it.
struct Derived2Layout {
    uint64_t B;  // radix buckets (0 in list mode)
    size_t off_rank, off_rdx, off_ioff, bytes;
};
Derived2Layout derived2_layout(uint64_t N, uint64_t L, bool list_mode);
int build_derived(lc_column* col, cudaStream_t st);

int decode_range(const lc_column* col, uint64_t begin, uint64_t count, void* out, cudaStream_t st);
int decode_ranges(const lc_column* col, const uint64_t* begin, const uint64_t* count,
                  const uint64_t* out_off, uint64_t m, void* out, uint64_t out_cap, cudaStream_t st);
int decode_ranges_noalloc(const lc_column* col, const uint64_t* begin, const uint64_t* count,
                          const uint64_t* out_off, uint64_t m, void* out, uint64_t out_cap, cudaStream_t st);
int access(const lc_column* col, const uint64_t* idx, uint64_t m, void* out, cudaStream_t st);
int set_query_plan(int plan);  // lc_set_query_plan
int lower_bound(const lc_column* col, const void* v, uint64_t m, uint64_t* out, cudaStream_t st);
int quantile(const lc_column* col, const uint64_t* ks, uint64_t m, uint64_t q, int exact, void* out, cudaStream_t st);
int decode_approx(const lc_column* col, uint64_t begin, uint64_t count, void* out, cudaStream_t st);
int set_op(bool is_and, const lc_column* a, int64_t la, const lc_column* b, int64_t lb, void* out, uint64_t cap,
           uint64_t* count, cudaStream_t st);

// Serving: one batch of requests over several columns (lc_query.cu).
int serve_launch(const ColView* views_d, int key_bytes, const SrvReq* qreqs_d, uint32_t nqreq, uint64_t nq,
                 const uint64_t* qin_d, uint64_t* qout_d, const SrvReq* dreqs_d, uint32_t ndreq,
                 const uint64_t* work_off_d, uint64_t nwork, uint32_t max_tile_segs, uint32_t* status_d,
                 cudaStream_t st);
uint64_t tile_of_key(const lc_column* col, uint64_t i);

// Exclusive scan of n uint32 counts into n+1 uint64 offsets (out[n] = total),
// optionally applying f(count) = even_words(count bits) first.
enum class ScanOp { Identity, BitsToEvenWords };
// scan_exclusive's tile: kScanThreads x kScanItems values per CTA, one
// uint64 partial per tile in tmp (scan_tmp_bytes).
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;
int scan_exclusive(const uint32_t* in, uint64_t* out, uint64_t n, ScanOp op, void* tmp,
                   size_t tmp_bytes, cudaStream_t st);
size_t scan_tmp_bytes(uint64_t n);

int cuda_status(cudaError_t e);

// Per-device set-up (kernel attributes, constant tables) done once per device
// and process.  Thread-safe; a set-up that fails is tried again on the next
// call.  Use one DeviceOnce object per set-up step, at namespace scope.
constexpr int kMaxDevices = 64;
struct DeviceOnce {
    std::mutex mu;
    std::atomic<bool> done[kMaxDevices];
};
template <typename F>
int once_per_device(DeviceOnce& o, F&& f) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LC_ERR_INTERNAL;
    if (o.done[dev].load(std::memory_order_acquire)) return LC_OK;
    std::lock_guard<std::mutex> lk(o.mu);
    if (o.done[dev].load(std::memory_order_relaxed)) return LC_OK;
    const int rc = f();
    if (rc == LC_OK) o.done[dev].store(true, std::memory_order_release);
    return rc;
}
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per device.
template <typename K>
int smem_attr_once(DeviceOnce& o, K* kernel, size_t bytes) {
    return once_per_device(o, [&] {
        return cuda_status(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    });
}

// Small host <-> device transfers (descriptors, headers, counts) made by
// kernels on page-locked mapped host memory instead of by the copy engines,
// so that they never queue behind a caller's large copies on other streams.
// The staging memory is per host thread and device; a region stays in use
// until the stream is synchronised with stage_sync.
//   stage_h2d: bytes from src_host to dst_dev, ordered on st (above 1 MB by
//              an ordinary copy).  src_host may be reused on return.
//   stage_d2h: bytes from src_dev; *host_out points at them once stage_sync(st)
//              has returned.
int stage_h2d(void* dst_dev, const void* src_host, size_t bytes, cudaStream_t st);
int stage_d2h(const void* src_dev, size_t bytes, cudaStream_t st, const void** host_out);
int stage_sync(cudaStream_t st);

// lc_selftest_wait: the decoders' bounded mbarrier wait on a barrier nobody
// completes, limited to `polls` polls.
int wait_selftest(uint32_t polls, cudaStream_t st);

// Count of kernel launches issued by the library in this process.
void note_launch(uint32_t k = 1);

// Tracing (lc_timing_enable): brackets one launch with CUDA events on its
// stream when tracing is on.  Use as { KTime kt("name", st); kernel<<<...>>>(); }
struct KTime {
    KTime(const char* name, cudaStream_t st);
    ~KTime();
    const char* name;
    cudaStream_t st;
    cudaEvent_t a, b;
};

// Host wall time of a phase of a call (reported by lc_timing_read under
// "host:<name>", synchronisations included), recorded while tracing is on.
struct HTime {
    explicit HTime(const char* name);
    ~HTime();
    const char* name;
    double t0;
};

}  // namespace lcx
