/*
 * lc.h -- C ABI of the GB300 learned compressor for sorted integer keys
 * (arXiv 2412.10770, "Learned Data Compression: Challenges and Opportunities
 * for the Future").
 *
 * Problem contract (Def. 1, Sec. I): given sorted keys K[0..N), build a compact
 * encoding K^c and a decoder with Dec(K^c)[i] = K[i] for every i; the
 * compression ratio is r = size(K^c) / size(K).
 *
 * Model (Def. 2, Eq. (1), Sec. II-A): an eps-PLA f whose segments
 * (s_j, alpha_j, beta_j) keep |K[i] - floor(f(i))| <= eps, stored with the
 * residuals Delta[i] = K[i] - floor(f(i)) (Sec. I, Fig. 2).  This library's
 * reading:
 *   - segments are anchored (beta_j = K[s_j]) with an int64 Q32 slope M_j;
 *     floor(f(i)) = K[s_j] + floor(M_j (i - s_j) / 2^32) in exact integer
 *     arithmetic (128-bit product, arithmetic shift);
 *   - they come from a greedy shrinking-cone fit inside fixed chunks of
 *     2^chunk_log2 keys (the paper's O'Rourke fit, Sec. II-A, is replaced);
 *     the slope is the floor midpoint of the final cone (0 for one key);
 *   - residuals are zigzag-coded and bit-packed LSB-first at a width chosen per
 *     segment, w_j <= ceil(log2(2 eps + 1)) (Sec. II-A); the anchor's residual
 *     (always 0) is not stored;
 *   - the byte layout "LCF1" is identical on the CPU and the GPU: a 64-byte
 *     header, the chunk directory (key, segment and payload-word offsets), the
 *     per-segment model (intercept, slope, bit offset, start, width) and the
 *     payload words.  lc_serialize returns exactly these bytes.
 *
 * Conventions
 *   - Every function returns an int status: LC_OK (0) or a negative LC_ERR_*.
 *     No function throws, aborts, or prints.
 *   - "_dev" pointers are device memory owned by the caller; they must stay
 *     valid until the work queued on `stream` has finished.  "host" pointers
 *     are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls are asynchronous on it unless marked "synchronous".
 *   - Keys are unsigned integers of key_bytes = 4 or 8 bytes, little-endian.
 *   - An lc_column owns its device memory; free it with lc_free.  A column may
 *     be read (decode, access, lower_bound) from several streams at once.
 *   - Device memory comes from the device's default stream-ordered pool
 *     (cudaMallocAsync).  The first lc_compress / lc_compress_batch /
 *     lc_deserialize on a device raises that pool's release threshold to an
 *     eighth of the device's memory (at least 8 GiB), so that freed blocks up
 *     to that size stay mapped for the next column instead of being handed
 *     back to the CUDA driver at every synchronisation.
 *   - Device-side errors (an index >= N in lc_access) are recorded in the
 *     column's status word and reported by lc_status.
 */
#ifndef LC_H
#define LC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LC_OK = 0,
    LC_ERR_INVALID_ARG = -1,  /* null pointer, key_bytes not 4/8, eps > 2^30, chunk_log2 not in [8,16] */
    LC_ERR_UNSORTED = -2,     /* keys are not non-decreasing */
    LC_ERR_OUT_OF_RANGE = -3, /* index >= N, or begin + count > N */
    LC_ERR_NOMEM = -4,        /* device or host allocation failed */
    LC_ERR_CORRUPT = -5,      /* lc_deserialize: bytes are not a valid LCF1 blob */
    LC_ERR_CUDA = -6,         /* a CUDA runtime call failed */
    LC_ERR_TIMEOUT = -7,      /* a bounded device or host wait gave up */
    LC_ERR_BUSY = -8,         /* serving: no slot or HBM budget free right now */
    LC_ERR_UNSUPPORTED = -10, /* operation not defined for this column (lower_bound on a list column) */
    LC_ERR_INTERNAL = -9,
    LC_ERR_STALE = -11        /* a replayed batch graph met keys whose K^c does not fit its plan */
};

typedef struct lc_column lc_column;

/* Fit parameters.  eps: the error bound of Def. 2, 0 <= eps <= 2^30.
 * chunk_log2: log2 of the chunk length in keys, 8..16 (16 by default).
 * span_log2: log2 of the keys each speculating GPU thread of the fit walks,
 * 5, 6 or 7 (0: the default, 6); a launch parameter only: K^c is the same for
 * every value. */
typedef struct {
    uint64_t eps;
    uint32_t chunk_log2;
    uint32_t span_log2;
} lc_params;

/* Header facts of a column (synchronous, host-side copy). */
typedef struct {
    uint64_t n;          /* keys */
    uint64_t chunks;     /* C */
    uint64_t segments;   /* L, the number of eps-PLA segments */
    uint64_t words;      /* W, 64-bit payload words */
    uint64_t lists;      /* lists in list mode, 0 for one column */
    uint64_t bytes;      /* size(K^c) in bytes (Def. 1) */
    uint64_t eps;        /* eps (0 in list mode) */
    uint32_t key_bytes;  /* 4 or 8 */
    uint32_t chunk_log2; /* 0 in list mode */
} lc_info_t;

/* ------------------------------------------------------------ compression */

/* K^c of one sorted column (Def. 1 encoding stage; Def. 2; Fig. 2 encoding).
 * keys_dev: n keys of key_bytes bytes, non-decreasing, device memory, not
 * modified.  params may be NULL (eps = 0, chunk_log2 = 16).  On success *out
 * is a new column.  Synchronous with respect to `stream`: it returns once the
 * column is complete (the totals of segments and payload words are read back
 * to size the allocation).  LC_ERR_UNSORTED if a key is smaller than its
 * predecessor. */
int lc_compress(const void* keys_dev, uint64_t n, int key_bytes, const lc_params* params,
                void* stream, lc_column** out);

/* lc_compress with the "jump" fit in place of the greedy, aiming at Sec.
 * II-A's objective of the fewest segments (the one O'Rourke's algorithm
 * reaches for free lines).  Every feasible anchored segment is a prefix of the
 * greedy one from its anchor, so with r(p) = the greedy's next anchor from p
 * (taken up to 96 keys; "long" beyond), the segment from anchor a ends at the
 * position in (a, r(a)] whose own r reaches farthest (long counts as
 * farthest; ties: the first position): the fewest segments whenever no
 * segment exceeds 96 keys.  An anchor whose greedy segment is long keeps that
 * segment, and a chunk keeps the jump segmentation only if it has fewer
 * segments than the greedy's, so a column never has more.  Slopes, widths and
 * the byte format are those of lc_compress; every query works unchanged.
 * Same arguments, errors and synchronisation as lc_compress; costs one more
 * walk of up to 96 keys per key. */
int lc_compress_jump(const void* keys_dev, uint64_t n, int key_bytes, const lc_params* params,
                     void* stream, lc_column** out);

/* K^c of many sorted lists stored back to back (inverted-index posting lists,
 * Sec. III-A).  ids_dev: all keys, device memory.  list_begin: nlists+1
 * non-decreasing offsets (host memory), list l is ids[list_begin[l],
 * list_begin[l+1]), each list non-decreasing on its own.  eps and chunk_log2:
 * one entry per list (host memory), or NULL for 0 and 16.  Every list is
 * compressed as its own column (chunks restart at each list), all lists in
 * one launch of each kernel.  span_log2: as in lc_params (0: default), one
 * value for the batch.  Synchronous like lc_compress. */
int lc_compress_batch(const void* ids_dev, const uint64_t* list_begin, uint64_t nlists,
                      int key_bytes, const uint64_t* eps, const uint8_t* chunk_log2, uint32_t span_log2,
                      void* stream, lc_column** out);

/* The batching path as one CUDA graph.  lc_batch_create compresses the lists
 * once, as lc_compress_batch does (synchronously), which fixes the column's
 * layout (segments, payload words, decode tiles).  It then records into one
 * CUDA graph every step of that compress (speculation, chain, segment models
 * and widths, bit offsets, packing, the derived directories) writing into the
 * same column, followed by a decode of every list into out_dev (device, N keys
 * of key_bytes).  lc_batch_launch replays the graph on `stream` with no host
 * synchronisation: the lists in ids_dev are compressed again and decoded.
 * For the same ids the column's bytes are those of lc_compress_batch.  The
 * graph checks on the device that the replay's segment and payload-word
 * totals equal the plan's; if not, the steps after the check do nothing,
 * lc_status on the column returns LC_ERR_STALE, and the column must be freed
 * (re-plan with lc_batch_create).  ids_dev and out_dev must outlive the
 * batch; lc_batch_column returns the column (owned by the batch, freed by
 * lc_batch_free).  Same arguments and errors as lc_compress_batch. */
typedef struct lc_batch lc_batch;
int lc_batch_create(const void* ids_dev, const uint64_t* list_begin, uint64_t nlists, int key_bytes,
                    const uint64_t* eps, const uint8_t* chunk_log2, uint32_t span_log2, void* out_dev, void* stream,
                    lc_batch** out);
int lc_batch_launch(lc_batch* batch, void* stream);
const lc_column* lc_batch_column(const lc_batch* batch);
void lc_batch_free(lc_batch* batch);

/* ------------------------------------------------------------ decoding */

/* Dec(K^c)[begin .. begin+count) (Fig. 2 decoding stage:
 * K[i] = floor(f_j(i)) + Delta[i]) into out_dev (count keys of key_bytes
 * bytes, device memory).  The full column is (0, N); in list mode list l is
 * (list_begin[l], list_begin[l+1] - list_begin[l]).  Asynchronous.
 * LC_ERR_OUT_OF_RANGE if begin + count > N; LC_ERR_INVALID_ARG if out_dev is
 * not a multiple of key_bytes (here and in lc_decode_ranges*). */
int lc_decode(const lc_column* col, uint64_t begin, uint64_t count, void* out_dev, void* stream);

/* Several ranges in one launch: range r is keys [begin[r], begin[r] +
 * count[r]) written to out_dev at out_off[r] keys.  begin_dev, count_dev and
 * out_off_dev are device arrays of m uint64 values; out_dev holds out_cap keys.
 * Both are validated on the device: a range past N, or one whose output
 * [out_off[r], out_off[r] + count[r]) does not fit in out_cap keys, is
 * recorded in the status word (LC_ERR_OUT_OF_RANGE) and skipped.
 * Asynchronous. */
int lc_decode_ranges(const lc_column* col, const uint64_t* begin_dev, const uint64_t* count_dev,
                     const uint64_t* out_off_dev, uint64_t m, void* out_dev, uint64_t out_cap, void* stream);

/* lc_decode_ranges for callers that cannot allocate device memory.  It takes
 * the same arguments, does the same work and writes the same output, but calls no cudaMalloc, cudaFree
 * or allocating library routine.  This helps callers whose request path must
 * not allocate: a serving loop that has to keep the allocator, and the device
 * synchronisation a cudaFree can cause, out of its latency; or an application
 * that owns all device memory and hands libraries only its own buffers.  The
 * paper has no counterpart: this is an interface choice of the library.
 *   - m <= LC_NOALLOC_MAX_RANGES, else LC_ERR_INVALID_ARG (nothing launched).
 *   - The work lists live in one file-scope device array of about 0.7 MB that
 *     every GPU loading the library keeps until the process exits.
 *   - The first call on a device looks up that array's device address (with
 *     the device current) and caches it; make this first call before any
 *     stream capture.
 *   - All calls share the array and leave their work lists in it.  Calls on
 *     one stream are ordered and safe; calls whose kernels overlap on the GPU
 *     (other streams, other host threads) race on it. */
#define LC_NOALLOC_MAX_RANGES 32768
int lc_decode_ranges_noalloc(const lc_column* col, const uint64_t* begin_dev, const uint64_t* count_dev,
                             const uint64_t* out_off_dev, uint64_t m, void* out_dev, uint64_t out_cap,
                             void* stream);

/* Every key of every list (list mode) or of the column.  Same as
 * lc_decode(col, 0, N, ...). */
int lc_decode_batch(const lc_column* col, void* out_dev, void* stream);

/* A decode recorded once into a CUDA graph and replayed (the batching path:
 * every list of a batch column decoded by one persistent launch).  The graph
 * holds lc_decode(col, begin, count, out_dev); col and out_dev must outlive it.
 * Recording uses `stream` (a non-default stream; NULL records on a private
 * stream).  lc_graph_launch replays it asynchronously on `stream`. */
typedef struct lc_graph lc_graph;
int lc_graph_decode(const lc_column* col, uint64_t begin, uint64_t count, void* out_dev, void* stream,
                    lc_graph** out);
int lc_graph_launch(lc_graph* graph, void* stream);
void lc_graph_free(lc_graph* graph);

/* Rank access (Sec. III-C, the quantile query f(i) + Delta[i]): out[q] =
 * K[idx[q]] for q < m.  idx_dev: m uint64 indices (device).  out_dev: m keys
 * of key_bytes bytes (device).  An index >= N yields 0 and sets
 * LC_ERR_OUT_OF_RANGE in the status word.  Asynchronous. */
int lc_access(const lc_column* col, const uint64_t* idx_dev, uint64_t m, void* out_dev,
              void* stream);

/* How lc_access and lc_lower_bound (and their _host forms) run a batch; the
 * results do not depend on it.
 *   LC_QUERIES_DIRECT: one query per thread, in the caller's order: each
 *     query's dependent loads (rank word or radix entry, 32-byte record,
 *     payload words) go to DRAM once the column's directories and payload
 *     exceed the L2 cache.
 *   LC_QUERIES_PARTITIONED: the queries are first sorted into buckets by the
 *     part of the column they read (key index for access; for lower_bound,
 *     the value against the keys at multiples of N/B), each bucket's slice of
 *     the directories and payload being about 16 MB; the buckets then run in
 *     order, so that their slices are read from L2, and the results are
 *     returned to query order.  Three launches (a per-tile counting sort, the
 *     lookups bucket by bucket, the gather) and 10 bytes per query of
 *     stream-ordered scratch (LC_ERR_NOMEM if the pool has none).
 *   LC_QUERIES_DECODED: the column is first decoded whole (one bulk decode
 *     into N keys of stream-ordered scratch), then the queries run
 *     partitioned against the decoded keys: an access reads its key there, a
 *     lower_bound finds its segment through the directories and searches the
 *     segment's decoded keys.  For dense batches (m comparable to N).
 *   LC_QUERIES_AUTO (the default): lc_access decoded when m >= 2^21,
 *     m >= N/8 and the keys take at least 64 MB; else partitioned when
 *     m >= 2^21, the column's records and rank words are at least 96 MB, and
 *     there is at least one query per 32 bytes of directories and payload;
 *     else direct.  lc_lower_bound direct (its lookups are bound by
 *     instruction issue; searching decoded keys is a chain of dependent
 *     loads).
 * Batches of 2^32 queries or more run direct.  Process-wide.  Returns the
 * previous setting, or LC_ERR_INVALID_ARG. */
enum { LC_QUERIES_AUTO = 0, LC_QUERIES_DIRECT = 1, LC_QUERIES_PARTITIONED = 2, LC_QUERIES_DECODED = 3 };
int lc_set_query_plan(int plan);

/* Value lower_bound through the segment directory (Sec. III-A segment
 * pruning, Table 2 binary search over segments): out[q] = first i with
 * K[i] >= v[q], or N when every key is smaller.  v_dev: m values of key_bytes
 * bytes (device).  out_dev: m uint64 (device).  Single columns only
 * (LC_ERR_UNSUPPORTED in list mode).  Asynchronous. */
int lc_lower_bound(const lc_column* col, const void* v_dev, uint64_t m, uint64_t* out_dev,
                   void* stream);

/* End to end from host memory: the calls above with their inputs and
 * outputs in host memory.  The library copies them to and from device
 * buffers it takes from the stream-ordered pool and releases in the order of
 * `stream`; with page-locked ("pinned") host memory every copy is
 * asynchronous on `stream`, so that calls on several streams overlap their
 * copies with one another's kernels (with pageable memory the copies are
 * synchronous).  Host buffers must stay valid, and outputs unread, until the
 * work queued on `stream` has finished.
 *   lc_compress_host: keys_host as lc_compress's keys_dev; synchronous like
 *     lc_compress (the column is complete on return).
 *   lc_decode_host: Dec(K^c)[begin .. begin+count) into out_host.
 *   lc_decode_ranges_host: begin/count/out_off (m uint64 each) in host
 *     memory; out_host holds out_cap keys and is copied back whole.
 *   lc_access_host, lc_lower_bound_host: m queries in, m results out.
 * Errors as the device calls. */
int lc_compress_host(const void* keys_host, uint64_t n, int key_bytes, const lc_params* params, void* stream,
                     lc_column** out);
int lc_decode_host(const lc_column* col, uint64_t begin, uint64_t count, void* out_host, void* stream);
int lc_decode_ranges_host(const lc_column* col, const uint64_t* begin_host, const uint64_t* count_host,
                          const uint64_t* out_off_host, uint64_t m, void* out_host, uint64_t out_cap, void* stream);
int lc_access_host(const lc_column* col, const uint64_t* idx_host, uint64_t m, void* out_host, void* stream);
int lc_lower_bound_host(const lc_column* col, const void* v_host, uint64_t m, uint64_t* out_host, void* stream);

/* Quantiles (Sec. III-C, Table 2): out[r] = the k[r]-th q-quantile of the
 * column, the key at index floor(N k / q) (the last key for k = q; the index
 * is computed exactly).  exact = 1: f(i) + Delta[i], the key itself (rank
 * access).  exact = 0: floor(f(i)) from the segments alone, without reading
 * any residual (approximate query processing; within eps of the key, Def. 2).
 * k_dev: m uint64 values (device), 0 <= k <= q; a k > q yields 0 and sets
 * LC_ERR_OUT_OF_RANGE in the status word.  out_dev: m keys (device).  q >= 1.
 * Single columns only (LC_ERR_UNSUPPORTED in list mode).  Asynchronous. */
int lc_quantile(const lc_column* col, const uint64_t* k_dev, uint64_t m, uint64_t q, int exact, void* out_dev,
                void* stream);

/* Segments-only decode (Sec. III-C approximate query processing): out_dev
 * receives floor(f(i)) for i in [begin, begin + count), each within eps of
 * K[i] (Def. 2); the residual array is not read.  Layout and errors as
 * lc_decode.  Asynchronous. */
int lc_decode_approx(const lc_column* col, uint64_t begin, uint64_t count, void* out_dev, void* stream);

/* Posting-list AND / OR (Sec. III-A, Fig. 4): the sorted values present in
 * both lists (lc_intersect) or in either (lc_union), each value once.  A list
 * is list la of column a (a list-mode column) or, for la < 0, the whole of a
 * single column; likewise lb of b.  Both sides must have the same key_bytes.
 * The intersection looks every key of the shorter list up in the longer one
 * through the longer list's segment intercepts: each segment's key range is
 * known from its intercept and the next one, so only the one segment that
 * can hold the key is decoded (segment-level pruning in place of skip
 * pointers).  The union merges both decoded lists.
 *   out_dev: cap keys of key_bytes (device).  *count receives the result's
 *   length; if it exceeds cap, LC_ERR_INVALID_ARG is returned and nothing is
 *   written.  LC_ERR_OUT_OF_RANGE for a list index past the column's lists,
 *   LC_ERR_INVALID_ARG for la/lb < 0 on a list-mode column.  Synchronous. */
int lc_intersect(const lc_column* a, int64_t la, const lc_column* b, int64_t lb, void* out_dev, uint64_t cap,
                 uint64_t* count, void* stream);
int lc_union(const lc_column* a, int64_t la, const lc_column* b, int64_t lb, void* out_dev, uint64_t cap,
             uint64_t* count, void* stream);

/* Per-chunk cost of a column (Sec. II-A size of the model and residuals,
 * restated per chunk): out_host[c] = segments_c (key_bytes + 15) + 8 words_c
 * + 24, the bytes chunk c adds to K^c (its segments, payload words and chunk
 * directory entries; alignment padding excluded).  cap >= C entries (host
 * memory).  Used to choose eps per partition (Sec. IV-A).  Synchronous. */
int lc_chunk_bytes(const lc_column* col, uint64_t* out_host, uint64_t cap);

/* Scalar conveniences (synchronous, legacy default stream). */
int lc_access1(const lc_column* col, uint64_t i, uint64_t* key);
int lc_lower_bound1(const lc_column* col, uint64_t v, uint64_t* pos);

/* ------------------------------------------------------------ serving */

/* Continuous batching over device-resident columns.  A server keeps `slots`
 * CUDA streams; a scheduler thread takes requests as they are submitted and,
 * whenever a slot is free, packs the waiting requests that fit in the free
 * HBM budget (device memory for their inputs and outputs) into one batch:
 * one fused launch for all access and lower_bound requests (over any of the
 * columns), one persistent launch for all range decodes, with the copies in
 * and out on the same stream.  Batches on different slots overlap on the
 * device; a request that arrives while others run is admitted as soon as a
 * slot and its memory are free.  Results equal those of the single-request
 * calls (lc_access, lc_lower_bound, lc_decode).  The paper has no serving
 * layer; this is the library's runtime around its queries (Sec. III). */
enum { LC_OP_ACCESS = 1, LC_OP_LOWER_BOUND = 2, LC_OP_DECODE = 3 };

typedef struct {
    uint32_t op;       /* LC_OP_* */
    uint32_t column;   /* index into the server's columns */
    uint64_t count;    /* ranks, values, or keys to decode */
    uint64_t begin;    /* LC_OP_DECODE: first key */
    const void* input; /* host: count uint64 ranks (access) or count values of key_bytes (lower_bound) */
    void* output;      /* host: count keys (access, decode) or count uint64 positions (lower_bound);
                          page-locked memory lets the copy overlap */
    uint64_t user;     /* returned in the completion */
} lc_request;

typedef struct {
    uint64_t ticket;
    uint64_t user;
    int32_t status;      /* LC_OK, or LC_ERR_OUT_OF_RANGE / LC_ERR_NOMEM (larger than the whole budget) / ... */
    uint32_t batch_size; /* requests in the batch it ran in */
    double latency_us;   /* from lc_server_submit to completion */
} lc_completion;

typedef struct {
    uint64_t submitted, completed, batches;
    uint64_t peak_hbm_bytes;    /* most device memory held by batches at once (<= budget) */
    uint32_t peak_inflight;     /* most batches on the device at once */
    uint32_t slots;
    double launch_us_max;     /* longest host time spent packing and launching one batch */
    double launch_us_total;   /* host time spent packing and launching, all batches */
    uint64_t staging_regrows; /* page-locked staging buffers grown (each synchronises the device) */
} lc_server_stats_t;

typedef struct lc_server lc_server;

/* cols: ncols single-mode or list-mode columns of one key width, all on the
 * current device; they must outlive the server.  hbm_budget: bytes of device
 * memory the server may hold for request inputs and outputs; memory a batch
 * frees stays reserved in the server's own pool until lc_server_destroy.  slots: streams
 * (batches in flight), 1..64. */
int lc_server_create(lc_column* const* cols, int ncols, uint64_t hbm_budget, int slots, lc_server** out);
/* Queue one request (thread-safe, non-blocking).  The input and output
 * buffers must stay valid until its completion has been returned. */
int lc_server_submit(lc_server* server, const lc_request* req, uint64_t* ticket);
/* Up to `max` finished requests, without waiting. */
int lc_server_poll(lc_server* server, lc_completion* out, int max, int* got);
/* Up to `max` finished requests, waiting at most timeout_us for the first. */
int lc_server_wait(lc_server* server, lc_completion* out, int max, int* got, uint64_t timeout_us);
int lc_server_stats(lc_server* server, lc_server_stats_t* stats);
/* Finish the queued and running work, then release the server. */
int lc_server_destroy(lc_server* server);

/* The plain path: one request alone, synchronously (copy in, one kernel, copy
 * out, wait) on `stream`. */
int lc_serve_sync(lc_column* const* cols, int ncols, const lc_request* req, void* stream, lc_completion* out);

/* ------------------------------------------------------------ baseline codec */

/* Frame-of-reference delta bit-packing in blocks of 128 keys ("FOR1"), the
 * conventional codec the learned compressor is compared against in the scale
 * sweep (the paper compares against such codecs in Sec. II-C, Fig. 3a).  Not
 * part of the learned method.  Block b stores its first key, the bit length
 * w_b of its largest gap, and its 128 gaps K[128b+i] - K[128b+i-1] (gap 0 is 0,
 * gaps past N are 0) at w_b bits each, LSB-first in 4 w_b 32-bit words; block b
 * starts at word 4 (w_0 + ... + w_{b-1}).  Layout: a 32-byte header ("FOR1",
 * key_bytes u32, N u64, B u64 blocks, W u64 payload words), block_base
 * (key_bytes x B), block_width (u8 x B), payload (u32 x W), each array 16-byte
 * aligned with zero padding.
 *   lc_for_compress: keys_dev as in lc_compress (device, non-decreasing, not
 *     modified); synchronous; LC_ERR_UNSORTED if a key is below its
 *     predecessor.  *out owns its device memory (lc_for_free).
 *   lc_for_decode: all N keys into out_dev (device, N x key_bytes);
 *     asynchronous on `stream`.
 *   lc_for_size / lc_for_serialize: the exact FOR1 bytes (synchronous). */
typedef struct lc_for lc_for;
int lc_for_compress(const void* keys_dev, uint64_t n, int key_bytes, void* stream, lc_for** out);
int lc_for_decode(const lc_for* f, void* out_dev, void* stream);
int lc_for_size(const lc_for* f, uint64_t* bytes);
int lc_for_serialize(const lc_for* f, void* host, uint64_t cap, uint64_t* len);
void lc_for_free(lc_for* f);

/* ------------------------------------------------------------ size, bytes, status */

/* r = size(K^c) / size(K) with size(K) = N * key_bytes (Def. 1).  Returns a
 * negative value for a NULL column and 0 for N = 0.  Synchronous, host only. */
double lc_ratio(const lc_column* col);

/* size(K^c) in bytes.  Synchronous, host only. */
int lc_size(const lc_column* col, uint64_t* bytes);

int lc_info(const lc_column* col, lc_info_t* info);

/* Copy the exact K^c bytes (the LCF1 blob) into host memory.  cap: capacity
 * of `host`; *len receives the blob length (also when cap is too small, in
 * which case LC_ERR_INVALID_ARG is returned).  Synchronous. */
int lc_serialize(const lc_column* col, void* host, uint64_t cap, uint64_t* len);

/* Validate an LCF1 blob held in host memory and upload it as a new column.
 * LC_ERR_CORRUPT if any structural fact of the format fails.  Synchronous. */
int lc_deserialize(const void* host, uint64_t len, void* stream, lc_column** out);

/* Wait for `stream`, then return and clear the column's device-side status
 * (LC_OK or the first LC_ERR_* recorded by a kernel).  Synchronous. */
int lc_status(const lc_column* col, void* stream);

/* Check of the library's bounded device waits, with no fault and no hang: one
 * thread waits, for at most `polls` polls (1 .. 2^20), on an mbarrier that
 * nobody completes, the same wait the decoders use on their bulk copies
 * (there with a limit of 2^22 polls, after which a decode records
 * LC_ERR_TIMEOUT in the column's status word and stops).  Returns
 * LC_ERR_TIMEOUT when the wait gave up as designed, LC_OK if it completed
 * (never), LC_ERR_INVALID_ARG for a polls value out of range.  Synchronous. */
int lc_selftest_wait(uint32_t polls, void* stream);

/* Release the column.  lc_free first waits for the whole device;
 * lc_free_async releases the device memory in the order of `stream` instead,
 * so the host does not wait: every use of the column must be on `stream` or
 * already complete.  The handle is invalid after either call. */
void lc_free(lc_column* col);
int lc_free_async(lc_column* col, void* stream);

const char* lc_strerror(int status);

/* Version of the library (major * 10000 + minor * 100 + patch). */
int lc_version(void);

/* Diagnostics: kernels this process has launched through the library so far. */
uint64_t lc_launch_count(void);

/* Diagnostics: bytes of the current device's default stream-ordered memory
 * pool (where the library's per-call device buffers come from) in use now,
 * and the most in use at once since the high-water mark was last reset.
 * reset = 1 first resets that mark to the current use.  Either output may be
 * NULL.  Synchronous (host only). */
int lc_pool_usage(int reset, uint64_t* used_now, uint64_t* used_high);

/* Tracing: while enabled, every kernel the library launches is bracketed by
 * two CUDA events recorded on its own stream, and its device time is added to
 * a per-kernel total.  lc_timing_read waits for the recorded work, returns up
 * to `max` entries (name, launches, total milliseconds) and resets the totals.
 * Enabling costs two event records per launch. */
typedef struct {
    char name[40];
    uint64_t launches;
    double total_ms;
} lc_kernel_time;
int lc_timing_enable(int on);
int lc_timing_read(lc_kernel_time* out, int max, int* got);

#ifdef __cplusplus
}
#endif

#endif /* LC_H */
