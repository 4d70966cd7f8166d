// lc_query.cu -- decoding from K^c on the GPU: bulk and range decode, rank
// access and value lower_bound (Def. 1 decoding, Fig. 2 decoding stage
// K[i] = floor(f_j(i)) + Delta[i]; Table 2 / Sec. III-A segment search).
//
// Decode works on tiles of 2048 keys that never cross a chunk.  A persistent
// CTA copies a tile's rank words (segment starts as bits, with the count
// before), the records of every segment that meets it and its payload words
// into shared memory with bulk copies, two tiles in flight; every key then
// finds its segment by a rank (popcount): no search per key.  A thread
// decodes two neighbouring keys and stores them as one aligned vector, the
// warp's stores covering consecutive keys.  Access and lower_bound are
// dependent random loads from the same derived directories (rank words,
// 32-byte records, a radix table and 16/32-bit intercept offsets).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "lc_internal.h"
#include "lc_math.cuh"

namespace lcx {
namespace {

constexpr int kDecThreads = 128;
constexpr uint32_t kMaxSegsPerTile = kTile + 1;
constexpr uint32_t kRankPerTile = kTile / 64 + 1;  // rank words a tile's keys can touch
constexpr uint32_t kPayWords = kTile + 16;          // payload words a tile can need (32-bit)

// One stage of the decode pipeline in shared memory: the tile's rank words,
// the records of its segments (at most ms) and its payload window.
__host__ __device__ constexpr size_t dec_stage(uint32_t ms) {
    return (size_t)kRankPerTile * 16 + (size_t)ms * 32 + (size_t)kPayWords * 4;
}
// Shared memory of one decode CTA (two stages) when no tile meets more than
// ms segments.
__host__ __device__ constexpr size_t dec_smem(uint32_t ms) { return 2 * dec_stage(ms); }
constexpr size_t kDecSmem = dec_smem(kMaxSegsPerTile);
constexpr uint32_t kSpinLimit = 1u << 22;  // mbarrier polls before a decode gives up (seconds)

template <typename KT>
__device__ __forceinline__ uint64_t ld_icpt(const void* icpt, uint64_t j) {
    return (uint64_t)__ldg((const KT*)icpt + j);
}

// Tile index of key i (chunk-relative position `local` in chunk c).
__device__ __forceinline__ uint64_t tile_of(const ColView& v, uint64_t c, uint64_t local) {
    return v.chunk_tile_begin[c] + (local >> kTileLog);
}

// Chunk holding key i.
__device__ __forceinline__ uint64_t chunk_of(const ColView& v, uint64_t i) {
    if (!v.list_mode) return i >> v.chunk_log2;
    uint64_t lo = 0, hi = v.C - 1;  // last c with ckb[c] <= i
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(v.ckb + mid) <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------ decode pipeline
//
// A persistent CTA decodes a list of work items (a tile of 2048 keys, the
// wanted key range, the output).  Each tile's inputs are three contiguous runs
// of device memory, so thread 0 fetches them with bulk copies (TMA,
// cp.async.bulk) into one of two shared-memory stages, completing on that
// stage's mbarrier, while the CTA decodes the previous tile from the other
// stage: the rank words of the tile's keys, the 32-byte records of the
// segments that meet it, and the payload words its residuals occupy (the
// window precomputed in the tile directory, 16-byte aligned).  Every key then
// needs only shared memory: its segment from the rank word (anchors before +
// popcount), its model from the record, its residual from the payload window
// (Fig. 2 decoding stage, K[i] = floor(f_j(i)) + Delta[i]); 32 consecutive
// keys per warp, stored coalesced.

struct DecItem {
    uint64_t kbeg;     // first key of the tile (global index)
    uint64_t lo, hi;   // wanted keys [lo, hi) (global), clipped to the tile below
    uint64_t j0;       // first segment of the tile
    uint64_t r0;       // first rank word of the tile
    uint64_t pbit0;    // global bit of the payload window's first word
    void* out;         // output of key g: out[g - lo_key]
    uint64_t lo_key;
    uint32_t n;        // keys in the tile
    uint32_t ns;       // segments meeting the tile
    uint32_t ok;       // 0: nothing to decode (error or empty)
    uint32_t pad;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bounded wait for the phase with the given parity; false if it gave up
// after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kSpinLimit) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

struct DecStage {
    RankWord* rank;
    SegRec* rec;
    uint32_t* pay;
};

__device__ __forceinline__ DecStage dec_stage_at(uint8_t* smem, uint32_t ms, uint32_t s) {
    uint8_t* b = smem + s * dec_stage(ms);
    DecStage d;
    d.rank = (RankWord*)b;
    d.rec = (SegRec*)(b + kRankPerTile * 16);
    d.pay = (uint32_t*)(b + kRankPerTile * 16 + (size_t)ms * 32);
    return d;
}

// The decoders' bounded wait, made to run out: one thread waits on an
// mbarrier that expects one arrival which never comes, and records in
// *status whether the wait gave up (kStTimeout) or, impossibly, completed.
__global__ void wait_selftest_kernel(uint32_t* __restrict__ status, uint32_t polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *status = mbar_wait(&bar, 0u, polls) ? 0u : kStTimeout;
}

// Thread 0: fetch tile t of v into stage s; the item is written before the
// arrive, so that the waiting threads see it.  A tile that does not fit the
// stage (cannot happen: ms bounds every tile) or holds no wanted key is marked
// and its barrier completed without copies.
template <bool Approx = false>
__device__ void dec_issue(const ColView& v, uint64_t t, uint64_t lo_key, uint64_t hi_key, void* out, uint32_t ms,
                          const DecStage& sd, uint64_t* bar, DecItem* it) {
    const TileDesc td = v.tiles[t];
    DecItem d;
    d.kbeg = td.key_begin;
    d.n = td.n;
    d.lo = max(lo_key, td.key_begin);
    d.hi = min(hi_key, td.key_begin + td.n);
    d.j0 = td.seg_lo;
    d.r0 = td.key_begin >> 6;
    d.pbit0 = 32ull * td.pw0;
    d.out = out;
    d.lo_key = lo_key;
    const uint32_t ns = (uint32_t)(td.seg_hi - td.seg_lo + 1);
    const uint32_t nr = (uint32_t)(((td.key_begin + td.n - 1) >> 6) - d.r0 + 1);
    d.ns = ns;
    d.pad = 0;
    d.ok = d.lo < d.hi && ns <= ms && nr <= kRankPerTile && td.pwn <= kPayWords;
    *it = d;
    if (!d.ok) {
        if (ns > ms || nr > kRankPerTile || td.pwn > kPayWords) atomicOr(v.status, kStInternal);
        mbar_expect(bar, 0);
        return;
    }
    const uint32_t pwn = Approx ? 0u : td.pwn;  // the segments-only decode reads no payload
    mbar_expect(bar, nr * 16u + ns * 32u + pwn * 4u);
    bulk_load(sd.rank, v.rank + d.r0, nr * 16u, bar);
    bulk_load(sd.rec, v.recs + d.j0, ns * 32u, bar);
    if (pwn) bulk_load(sd.pay, v.pay32 + td.pw0, pwn * 4u, bar);
}

// Two keys stored as one aligned vector.
__device__ __forceinline__ void st_pair(uint64_t* p, uint64_t a, uint64_t b) {
    *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(a, b);
}
__device__ __forceinline__ void st_pair(uint32_t* p, uint32_t a, uint32_t b) {
    *reinterpret_cast<uint2*>(p) = make_uint2(a, b);
}

// All threads: the wanted keys of the item in stage sd.  Everything inside a
// tile is 32-bit: positions, segment offsets and payload bits relative to the
// tile (the low 32 bits of the global values suffice because every difference
// taken is below 2^32).
//
// A thread decodes two neighbouring keys p, p + 1 at once, starting where
// &out[p] is aligned to the pair: one rank word and one record serve both
// (key p + 1 only reads the next record when it starts a segment), their two
// residuals sit next to each other in one 64-bit window of the payload, and
// the pair goes out as one vector store.  An unpaired first or last key is
// decoded alone.  An anchor (t = 0) has no residual: its field is taken as 0.
template <typename KT, bool Approx = false>
__device__ __forceinline__ void dec_compute(const DecItem& d, const DecStage& sd) {
    const uint32_t p0 = (uint32_t)(d.lo - d.kbeg), p1 = (uint32_t)(d.hi - d.kbeg);
    KT* __restrict__ out = (KT*)d.out + (d.lo - d.lo_key) - p0;  // out[p]: key kbeg + p
    const uint32_t kb32 = (uint32_t)d.kbeg, koff = kb32 & 63u;
    const uint32_t j0 = (uint32_t)d.j0, pb0 = (uint32_t)d.pbit0, nsm1 = d.ns - 1;
    // pairs start at p = e (mod 2): there out + p is a multiple of 2 sizeof(KT)
    const uint32_t e = (uint32_t)(((uintptr_t)out / sizeof(KT)) & 1u);
    const uint32_t pa = p0 + ((p0 ^ e) & 1u);
    const uint32_t np = p1 > pa ? (p1 - pa) >> 1 : 0u;
    auto one = [&](uint32_t p) {
        const uint32_t g = kb32 + p;
        const RankWord rw = sd.rank[(koff + p) >> 6];
        const uint32_t jr = (uint32_t)rw.before - j0 + (uint32_t)__popcll(rw.bits << (63u - (g & 63u))) - 1u;
        const SegRec r = sd.rec[min(jr, nsm1)];  // the clamp only guards shared memory
        const uint32_t t = g - (uint32_t)r.kstart_w;
        const uint32_t w = (uint32_t)(r.kstart_w >> 56);
        const uint32_t lb = (uint32_t)r.bit1_n - pb0 + w * (t - 1u);
        const uint32_t q = min(lb >> 5, kPayWords - 2);
        const uint32_t z = Approx ? 0u : extract_bits(sd.pay[q], sd.pay[q + 1], lb & 31u, t ? w : 0u);
        out[p] = (KT)(r.icpt + (uint64_t)(line_at(r.slope, t) + (int64_t)unzigzag32(z)));
    };
    if (threadIdx.x == kDecThreads - 1 && pa > p0 && p0 < p1) one(p0);
    if (threadIdx.x == kDecThreads - 2 && p1 > pa && ((p1 - pa) & 1u)) one(p1 - 1);
#pragma unroll 4
    for (uint32_t i = threadIdx.x; i < np; i += kDecThreads) {
        const uint32_t p = pa + 2 * i;
        const uint32_t g = kb32 + p, x = koff + p, x1 = x + 1;
        const RankWord rw = sd.rank[x >> 6];
        const uint32_t jr = (uint32_t)rw.before - j0 + (uint32_t)__popcll(rw.bits << (63u - (x & 63u))) - 1u;
        const uint64_t bits1 = (x1 & 63u) ? rw.bits : sd.rank[x1 >> 6].bits;  // the rank word of key p + 1
        const bool starts1 = (bits1 >> (x1 & 63u)) & 1u;                     // key p + 1 opens a segment
        const SegRec r = sd.rec[min(jr, nsm1)];
        const uint32_t t = g - (uint32_t)r.kstart_w;
        const uint32_t w = (uint32_t)(r.kstart_w >> 56);
        // the window starts at residual t (t >= 1), or at residual 1 for an anchor
        const uint32_t lb = (uint32_t)r.bit1_n - pb0 + w * (t ? t - 1u : 0u);
        const uint32_t q = min(lb >> 5, kPayWords - 3);
        const uint32_t sh = lb & 31u;
        uint32_t za = 0, zb = 0;
        if (!Approx) {
            const uint32_t a0 = sd.pay[q], a1 = sd.pay[q + 1], a2 = sd.pay[q + 2];
            const uint64_t win = ((uint64_t)__funnelshift_r(a1, a2, sh) << 32) | __funnelshift_r(a0, a1, sh);
            const uint64_t mask = (1ull << w) - 1ull;
            za = (uint32_t)(win & mask);
            zb = (uint32_t)((win >> w) & mask);
        }
        const KT v0 = (KT)(r.icpt + (uint64_t)(line_at(r.slope, t) + (int64_t)unzigzag32(t ? za : 0u)));
        KT v1;
        if (starts1)
            v1 = (KT)sd.rec[min(jr + 1u, nsm1)].icpt;
        else
            v1 = (KT)(r.icpt + (uint64_t)(line_at(r.slope, t + 1u) + (int64_t)unzigzag32(t ? zb : za)));
        st_pair(out + p, v0, v1);
    }
}

// The pipeline over work items w = blockIdx.x, blockIdx.x + gridDim.x, ...
// < total; src(w, &view, &tile, &lo, &hi, &out) describes item w and is
// called by all 32 lanes of warp 0 together.
template <typename KT, typename Src, bool Approx = false>
__device__ void dec_pipeline(uint64_t total, const Src& src, uint8_t* smem, uint32_t ms) {
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ DecItem s_item[2];
    const uint64_t w0 = blockIdx.x;
    if (w0 >= total) return;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0]);
        mbar_init(&s_bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const ColView* vv;
    uint64_t t, lo, hi;
    void* o;
    // warp 0 describes the items (src is warp-collective), thread 0 issues
    if (threadIdx.x < 32) {
        src(w0, &vv, &t, &lo, &hi, &o);
        if (threadIdx.x == 0)
            dec_issue<Approx>(*vv, t, lo, hi, o, ms, dec_stage_at(smem, ms, 0), &s_bar[0], &s_item[0]);
    }
    uint32_t k = 0;
    for (uint64_t w = w0; w < total; w += gridDim.x, ++k) {
        const uint32_t s = k & 1u;
        const uint64_t wn = w + gridDim.x;
        if (threadIdx.x < 32 && wn < total) {
            src(wn, &vv, &t, &lo, &hi, &o);
            if (threadIdx.x == 0)
                dec_issue<Approx>(*vv, t, lo, hi, o, ms, dec_stage_at(smem, ms, s ^ 1u), &s_bar[s ^ 1u],
                                  &s_item[s ^ 1u]);
        }
        const bool got = mbar_wait(&s_bar[s], (k >> 1) & 1u);
        if (__syncthreads_or(!got)) {
            // a copy never completed: record it, wait (bounded) for the other
            // stage's copies, and stop
            if (threadIdx.x < 32) {
                src(w, &vv, &t, &lo, &hi, &o);
                if (threadIdx.x == 0) {
                    atomicOr(vv->status, kStTimeout);
                    if (wn < total) mbar_wait(&s_bar[s ^ 1u], ((k + 1) >> 1) & 1u);
                }
            }
            __syncthreads();
            return;
        }
        const DecItem d = s_item[s];
        if (d.ok) dec_compute<KT, Approx>(d, dec_stage_at(smem, ms, s));
        __syncthreads();  // stage s is free for item k + 2
    }
}

template <typename KT>
struct WholeSrc {
    const ColView* v;
    uint64_t t0, begin, end;
    KT* out;
    __device__ void operator()(uint64_t w, const ColView** vv, uint64_t* t, uint64_t* lo, uint64_t* hi,
                               void** o) const {
        *vv = v;
        *t = t0 + w;
        *lo = begin;
        *hi = end;
        *o = out;
    }
};

// Persistent: tiles t0 .. t0 + nt - 1, keys [begin, end) into out[g - begin].
template <typename KT>
__global__ void __launch_bounds__(kDecThreads, 12) decode_kernel(ColView v, uint64_t t0, uint64_t nt, uint64_t begin,
                                                             uint64_t end, KT* __restrict__ out) {
    if (v.gate && *v.gate == 0) return;  // a batch replay that does not fit its plan
    extern __shared__ __align__(16) uint8_t smem[];
    dec_pipeline<KT>(nt, WholeSrc<KT>{&v, t0, begin, end, out}, smem, v.max_tile_segs);
}

// The last r in [0, n) with off[r] <= w, for non-decreasing off with
// off[0] <= w, found by the 32 lanes of a warp together: each round probes 32
// evenly spaced entries and keeps the span after the last one that is <= w,
// so 16384 ranges take three rounds of loads instead of fourteen dependent
// ones.  Call with all 32 lanes; every lane gets the result.
__device__ __forceinline__ uint64_t warp_last_le(const uint64_t* __restrict__ off, uint64_t n, uint64_t w) {
    const uint32_t lane = threadIdx.x & 31u;
    uint64_t a = 0, b = n;  // the answer lies in [a, b)
    while (b - a > 1) {
        const uint64_t step = (b - a + 31) >> 5;
        const uint64_t i = a + step * lane;
        const bool ok = i < b && __ldg(off + i) <= w;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, ok);  // a prefix of lanes; lane 0 (i = a) always
        a += step * (31u - __clz(bal));
        b = min(b, a + step);
    }
    return a;
}

// Segments-only decode (Sec. III-C, approximate query processing without the
// residuals): the decode pipeline over tiles t0 .. t0 + nt - 1 with every
// residual taken as 0, so out[g - begin] = floor(f(g)), within eps of K[g];
// no payload is read.
template <typename KT>
__global__ void __launch_bounds__(kDecThreads, 12) decode_approx_kernel(ColView v, uint64_t t0, uint64_t nt,
                                                                    uint64_t begin, uint64_t end,
                                                                    KT* __restrict__ out) {
    extern __shared__ __align__(16) uint8_t smem[];
    dec_pipeline<KT, WholeSrc<KT>, true>(nt, WholeSrc<KT>{&v, t0, begin, end, out}, smem, v.max_tile_segs);
}

// Work items of a multi-range decode: range r covers tiles
// [first[r], first[r] + ntiles[r]).
__global__ void range_tiles_kernel(ColView v, const uint64_t* __restrict__ begin, const uint64_t* __restrict__ count,
                                   const uint64_t* __restrict__ out_off, uint64_t out_cap, uint64_t m,
                                   uint64_t* __restrict__ first, uint32_t* __restrict__ ntiles) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m; r += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = begin[r], cnt = count[r], o = out_off[r];
        if (cnt == 0 || b > v.N || cnt > v.N - b || o > out_cap || cnt > out_cap - o) {
            if (cnt) atomicOr(v.status, kStOutOfRange);
            first[r] = 0;
            ntiles[r] = 0;
            continue;
        }
        const uint64_t e = b + cnt - 1;
        const uint64_t cb = chunk_of(v, b), ce = chunk_of(v, e);
        const uint64_t tb = tile_of(v, cb, b - __ldg(v.ckb + cb));
        const uint64_t te = tile_of(v, ce, e - __ldg(v.ckb + ce));
        first[r] = tb;
        ntiles[r] = (uint32_t)(te - tb + 1);
    }
}

template <typename KT>
struct RangesSrc {
    const ColView* v;
    const uint64_t *begin, *count, *out_off, *first, *work_off;
    uint64_t m;
    KT* out;
    __device__ void operator()(uint64_t w, const ColView** vv, uint64_t* t, uint64_t* lo, uint64_t* hi,
                               void** o) const {
        const uint64_t a = warp_last_le(work_off, m, w);  // the range that holds item w
        *vv = v;
        *t = first[a] + (w - work_off[a]);
        *lo = begin[a];
        *hi = begin[a] + count[a];
        *o = out + out_off[a];
    }
};

template <typename KT>
__global__ void __launch_bounds__(kDecThreads, 12)
decode_ranges_kernel(ColView v, const uint64_t* __restrict__ begin, const uint64_t* __restrict__ count,
                     const uint64_t* __restrict__ out_off, uint64_t m, const uint64_t* __restrict__ first,
                     const uint64_t* __restrict__ work_off, KT* __restrict__ out) {
    extern __shared__ __align__(16) uint8_t smem[];
    dec_pipeline<KT>(work_off[m], RangesSrc<KT>{&v, begin, count, out_off, first, work_off, m, out}, smem,
                     v.max_tile_segs);
}

constexpr uint64_t kKeyMask = (1ull << 56) - 1;

// L2 eviction priorities for the random lookups: directories that many queries
// share (rank words, intercept levels, seg_icpt) are marked evict_last, the
// per-query records and payload words evict_first, so that the streaming part
// does not push the shared part out of L2.
__device__ __forceinline__ uint64_t policy_keep() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_stream() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ ulonglong2 ld2_hint(const void* ptr, uint64_t pol) {
    ulonglong2 r;
    asm("ld.global.nc.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;" : "=l"(r.x), "=l"(r.y) : "l"(ptr), "l"(pol));
    return r;
}
__device__ __forceinline__ uint64_t ld64_hint(const void* ptr, uint64_t pol) {
    uint64_t r;
    asm("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r) : "l"(ptr), "l"(pol));
    return r;
}
__device__ __forceinline__ void st64_hint(void* ptr, uint64_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(ptr), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st32_hint(void* ptr, uint32_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(ptr), "r"(v), "l"(pol) : "memory");
}
// A query stream element (read once): L2 evict_first, so that streaming the
// queries and results does not push the shared directories out of L2.
template <typename T>
__device__ __forceinline__ uint64_t ld_stream(const T* p, uint64_t pol) {
    if (sizeof(T) == 8) {
        uint64_t r;
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(pol));
        return r;
    }
    if (sizeof(T) == 2) {
        uint16_t r;
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(r) : "l"(p), "l"(pol));
        return r;
    }
    static_assert(sizeof(T) == 8 || sizeof(T) == 4 || sizeof(T) == 2, "8-, 4- or 2-byte stream elements");
    uint32_t r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}
template <typename T>
__device__ __forceinline__ void st_stream(T* p, uint64_t v, uint64_t pol) {
    if (sizeof(T) == 8) st64_hint(p, v, pol);
    else st32_hint(p, (uint32_t)v, pol);
}
__device__ __forceinline__ uint32_t ld32_hint(const void* ptr, uint64_t pol) {
    uint32_t r;
    asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(ptr), "l"(pol));
    return r;
}

__device__ __forceinline__ uint32_t ld16_hint(const void* ptr, uint64_t pol) {
    uint16_t r;
    asm("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(r) : "l"(ptr), "l"(pol));
    return r;
}

// One 32-byte record in one 256-bit load (records are 32-byte aligned: the
// array starts the derived allocation): one L1 request per lane, not two.
__device__ __forceinline__ SegRec load_rec_hint(const SegRec* p, uint64_t pol) {
    uint64_t a, b, c, d;
    asm("ld.global.nc.L2::cache_hint.v4.u64 {%0, %1, %2, %3}, [%4], %5;"
        : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
        : "l"(p), "l"(pol));
    SegRec r;
    r.icpt = a;
    r.slope = (int64_t)b;
    r.kstart_w = c;
    r.bit1_n = d;
    return r;
}

// rec_key with the payload words read under an L2 policy.
__device__ __forceinline__ uint64_t rec_key_hint(const ColView& v, const SegRec& r, uint32_t t, uint64_t pol) {
    if (t == 0) return r.icpt;
    const uint32_t w = (uint32_t)(r.kstart_w >> 56);
    const int64_t line = line_at(r.slope, t);
    if (w == 0) return r.icpt + (uint64_t)line;
    const uint64_t pos = (r.bit1_n & kBitMask) + (uint64_t)w * (t - 1);
    const uint64_t wi = pos >> 5;
    const uint32_t lo = ld32_hint(v.pay32 + wi, pol);
    const uint32_t hi = wi + 1 < 2 * v.W ? ld32_hint(v.pay32 + wi + 1, pol) : 0u;
    return r.icpt + (uint64_t)(line + (int64_t)unzigzag32(extract_bits(lo, hi, (uint32_t)(pos & 31u), w)));
}

// Rank access: the segment of key i comes from one rank word (anchor bits +
// anchors before), its model from one 32-byte record, its residual from the
// payload: three dependent loads.  i < v.N.
__device__ __forceinline__ uint64_t access_one(const ColView& v, uint64_t i, uint64_t keep, uint64_t stream) {
    const ulonglong2 rw = ld2_hint(v.rank + (i >> 6), keep);
    const uint64_t j = rw.y + __popcll(rw.x & (~0ull >> (63u - (uint32_t)(i & 63u)))) - 1;
    const SegRec r = load_rec_hint(v.recs + j, stream);
    return rec_key_hint(v, r, (uint32_t)(i - (r.kstart_w & kKeyMask)), stream);
}

template <typename KT>
__global__ void access_kernel(ColView v, const uint64_t* __restrict__ idx, uint64_t m, KT* __restrict__ out) {
    const uint64_t keep = policy_keep(), stream = policy_stream();
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    // the next query's rank is loaded while this one's dependent loads run
    uint64_t in = q < m ? ld_stream(idx + q, stream) : 0;
    for (; q < m; q += step) {
        const uint64_t i = in;
        if (q + step < m) in = ld_stream(idx + q + step, stream);
        if (i >= v.N) {
            atomicOr(v.status, kStOutOfRange);
            out[q] = 0;
            continue;
        }
        st_stream(out + q, access_one(v, i, keep, stream), stream);
    }
}

// Value lower_bound: the first i with K[i] >= x (N if none).  The last
// segment whose intercept (its first key) is < x lies in the radix bucket of
// x, between rdx[q] - 1 and rdx[q+1] - 1: a binary search over that run of
// seg_icpt (usually one or two entries) finds it.  Then the segment's own line
// brackets the answer: every key lies within R = 2^(w-1) of floor(f), so keys
// before t < (dx - R)/s are < x and the key at t >= (dx + R + 1)/s is >= x
// (s = slope / 2^32, dx = x - intercept).  A binary search inside the bracket
// finishes.  Dependent loads: one table entry pair, the intercept run, one
// 32-byte record, the payload words of the bracket.
__device__ __forceinline__ uint64_t lower_bound_in_segment(const ColView& v, uint64_t x, uint64_t j, uint64_t stream);

// The last segment whose intercept (its first key) is < x, for kmin < x <= kmax.
template <typename KT>
__device__ __forceinline__ uint64_t segment_below(const ColView& v, uint64_t x, uint64_t keep) {
    const uint64_t q = (x - v.kmin) >> v.rdx_shift;
    uint64_t lo = min(ld64_hint(v.rdx + q, keep), v.L), hi = min(ld64_hint(v.rdx + q + 1, keep), v.L);
    if (v.ioff_bytes) {
        // count of intercepts < x within [rdx[q], rdx[q+1]): all of them lie in
        // bucket q, so their offsets from the bucket's first value compare as
        // the intercepts do, and the offsets array is a quarter of the size
        const uint32_t xo = (uint32_t)((x - v.kmin) & ((1ull << v.rdx_shift) - 1));
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            const uint32_t k = v.ioff_bytes == 2 ? ld16_hint((const uint16_t*)v.ioff + mid, keep)
                                                 : ld32_hint((const uint32_t*)v.ioff + mid, keep);
            if (k < xo) lo = mid + 1;
            else hi = mid;
        }
    } else {
        while (lo < hi) {  // count of intercepts < x, within [rdx[q], rdx[q+1])
            const uint64_t mid = (lo + hi) >> 1;
            const uint64_t k = sizeof(KT) == 8 ? ld64_hint((const uint64_t*)v.icpt + mid, keep)
                                               : (uint64_t)ld32_hint((const uint32_t*)v.icpt + mid, keep);
            if (k < x) lo = mid + 1;
            else hi = mid;
        }
    }
    return lo ? lo - 1 : 0;  // lo >= 1 for sorted keys: icpt[0] = kmin < x
}

template <typename KT>
__device__ __forceinline__ uint64_t lower_bound_one(const ColView& v, uint64_t x, uint64_t keep, uint64_t stream) {
    if (v.L == 0 || x <= v.kmin) return 0;
    if (x > v.kmax) return v.N;
    return lower_bound_in_segment(v, x, segment_below<KT>(v, x, keep), stream);
}

// The first key index of segment j or after it whose key is >= x, given
// that segment j's intercept is < x: its line brackets the answer (see
// lower_bound_one), a binary search inside the bracket finishes.
__device__ __forceinline__ uint64_t lower_bound_in_segment(const ColView& v, uint64_t x, uint64_t j, uint64_t stream) {
    const SegRec r = load_rec_hint(v.recs + j, stream);
    const uint64_t ks = r.kstart_w & kKeyMask;
    const uint32_t n = (uint32_t)(r.bit1_n >> 48) + 1u;
    uint32_t a = 1, b = n;  // first t in [1, n) with key(t) >= x, or n
    // The bracket is taken for short segments too: it usually leaves a few
    // indices, whose residuals then fit the register window below.  Single
    // precision with the fast reciprocal errs by about 2^-20 relative (four
    // conversions, two sums, the 2-ulp reciprocal, two products), under 0.1
    // index for t < 2^16: inside the bracket's 2-index margin.
    if (n > 2 && r.slope > 0) {
        const uint32_t w = (uint32_t)(r.kstart_w >> 56);
        // 64-bit integers go to float as two 32-bit halves: a 64-bit
        // conversion would take the slow double-precision pipe
        const uint64_t dx = x - r.icpt;
        const float s = (float)(uint32_t)((uint64_t)r.slope >> 32) +
                        (float)(uint32_t)r.slope * 2.3283064365386963e-10f;  // keys per index
        const float rs = __fdividef(1.0f, s);
        const float th = ((float)(uint32_t)(dx >> 32) * 4294967296.0f + (float)(uint32_t)dx) * rs;
        // |residual| <= 2^(w-1) for a w-bit zigzag code (w = 32 is legal: eps up to 2^30)
        const float half = w ? (float)(1u << (w - 1)) : 0.0f;
        const float dl = (half + 1.0f) * rs + 2.0f;
        const float fa = th - dl, fb = th + dl + 1.0f;
        a = fa <= 1.0f ? 1u : (fa >= (float)n ? n : (uint32_t)fa);
        b = fb <= 1.0f ? 1u : (fb >= (float)n ? n : (uint32_t)fb);
        if (a > b) a = b;
    }
    const uint32_t w = (uint32_t)(r.kstart_w >> 56);
    if (a < b && w) {
        // the residuals of the bracket usually lie in 8 payload words: two
        // 16-byte loads, and the search then runs on registers instead of a
        // load per probe.  Probes that read the payload first narrow a
        // bracket whose residuals do not fit one such window.
        const uint64_t bit1 = r.bit1_n & kBitMask;
        auto fits = [&](uint32_t lo_t, uint32_t hi_t) {
            const uint64_t q0 = (bit1 + (uint64_t)w * (lo_t - 1)) >> 5;      // word of residual lo_t
            const uint64_t q1 = (bit1 + (uint64_t)w * (hi_t - 1) - 1) >> 5;  // word of residual hi_t - 1's last bit
            const uint64_t base = q0 & ~3ull;
            return q1 + 1 < base + 8 && base + 8 <= 2 * v.W;
        };
        while (a < b && !fits(a, b)) {
            const uint32_t mid = (a + b) >> 1;
            if (rec_key_hint(v, r, mid, stream) < x) a = mid + 1;
            else b = mid;
        }
        if (a < b) {
            const uint64_t base = ((bit1 + (uint64_t)w * (a - 1)) >> 5) & ~3ull;
            const ulonglong2 u = ld2_hint(v.pay32 + base, stream), u2 = ld2_hint(v.pay32 + base + 4, stream);
            const uint32_t W0 = (uint32_t)u.x, W1 = (uint32_t)(u.x >> 32), W2 = (uint32_t)u.y,
                           W3 = (uint32_t)(u.y >> 32), W4 = (uint32_t)u2.x, W5 = (uint32_t)(u2.x >> 32),
                           W6 = (uint32_t)u2.y, W7 = (uint32_t)(u2.y >> 32);
            const uint64_t off = bit1 - 32 * base;  // mod 2^64: the positions below are in [0, 256)
            while (a < b) {
                const uint32_t mid = (a + b) >> 1;
                const uint32_t pos = (uint32_t)(off + (uint64_t)w * (mid - 1));
                // words k and k + 1 of the window (k = pos / 32 < 7), three levels of selects
                const uint32_t k = pos >> 5;
                const bool b2 = k & 4u, b1 = k & 2u, b0 = k & 1u;
                const uint32_t a0 = b2 ? W4 : W0, a1 = b2 ? W5 : W1, a2 = b2 ? W6 : W2, a3 = b2 ? W7 : W3;
                const uint32_t c0 = b1 ? a2 : a0, c1 = b1 ? a3 : a1, c2 = b1 ? (b2 ? W7 : W4) : a2;
                const uint32_t z = extract_bits(b0 ? c1 : c0, b0 ? c2 : c1, pos & 31u, w);
                const uint64_t key = r.icpt + (uint64_t)(line_at(r.slope, mid) + (int64_t)unzigzag32(z));
                if (key < x) a = mid + 1;
                else b = mid;
            }
        }
        return ks + a;
    }
    while (a < b) {  // w = 0: the keys lie on the line
        const uint32_t mid = (a + b) >> 1;
        if (rec_key_hint(v, r, mid, stream) < x) a = mid + 1;
        else b = mid;
    }
    return ks + a;
}

template <typename KT>
__global__ void __launch_bounds__(256, 6) lower_bound_kernel(ColView v, const KT* __restrict__ vals, uint64_t m,
                                                          uint64_t* __restrict__ out) {
    const uint64_t keep = policy_keep(), stream = policy_stream();
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    // the next query's value is loaded while this one's dependent loads run
    uint64_t xn = q < m ? ld_stream(vals + q, stream) : 0;
    for (; q < m; q += step) {
        const uint64_t x = xn;
        if (q + step < m) xn = ld_stream(vals + q + step, stream);
        st_stream(out + q, lower_bound_one<KT>(v, x, keep, stream), stream);
    }
}

// ------------------------------------------------------------------ quantiles and segments-only (approximate) keys

// floor(f_j(i)) of key i from the segments alone (Def. 2: within eps of K[i]):
// the rank word gives the segment, its record the anchored line; no residual
// is read.
__device__ __forceinline__ uint64_t predict_one(const ColView& v, uint64_t i, uint64_t keep, uint64_t stream) {
    const ulonglong2 rw = ld2_hint(v.rank + (i >> 6), keep);
    const uint64_t j = rw.y + __popcll(rw.x & (~0ull >> (63u - (uint32_t)(i & 63u)))) - 1;
    const SegRec r = load_rec_hint(v.recs + j, stream);
    return r.icpt + (uint64_t)line_at(r.slope, (uint32_t)(i - (r.kstart_w & kKeyMask)));
}

// Index of the k-th q-quantile (Sec. III-C): floor(N k / q), the last key for
// k = q.  Exact for every k <= q (128-bit product).
__device__ __forceinline__ uint64_t quantile_index(uint64_t N, uint64_t k, uint64_t q) {
    const unsigned __int128 t = (unsigned __int128)N * k / q;
    return t >= N ? N - 1 : (uint64_t)t;
}

// out[r] = the ks[r]-th q-quantile: K[floor(N k/q)] (exact = 1, Sec. III-C)
// or floor(f(floor(N k/q))) from the segments only (exact = 0, the
// approximate answer within eps).  k > q is out of range (0 and a status bit).
template <typename KT>
__global__ void quantile_kernel(ColView v, const uint64_t* __restrict__ ks, uint64_t m, uint64_t q, int exact,
                                KT* __restrict__ out) {
    const uint64_t keep = policy_keep(), stream = policy_stream();
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t kn = r < m ? ld_stream(ks + r, stream) : 0;  // the next query, loaded ahead
    for (; r < m; r += step) {
        const uint64_t k = kn;
        if (r + step < m) kn = ld_stream(ks + r + step, stream);
        if (k > q) {
            atomicOr(v.status, kStOutOfRange);
            out[r] = 0;
            continue;
        }
        const uint64_t i = quantile_index(v.N, k, q);
        out[r] = (KT)(exact ? access_one(v, i, keep, stream) : predict_one(v, i, keep, stream));
    }
}

// ------------------------------------------------------------------ posting-list AND / OR (Sec. III-A, Fig. 4)
//
// AND: every key x of the shorter list S is looked up in the longer list L by
// a binary search over L's segment intercepts (each segment's key range
// starts at its intercept and ends before the next one, so only the one
// segment that can hold x is touched: segment-level pruning, Fig. 4b) and its
// line bracket; x is kept iff that key equals x (and x is not a repeat of the
// key before it in S).  OR: a merge-path merge of both decoded lists, keeping
// each value once.  Both compact their flags with an exclusive scan.

// The first index in [k0, k1) of list L (segments [s0, s1)) whose key is >= x,
// or k1.
template <typename KT>
__device__ __forceinline__ uint64_t lower_bound_range(const ColView& v, uint64_t x, uint64_t s0, uint64_t s1,
                                                      uint64_t k0, uint64_t k1, uint64_t keep, uint64_t stream) {
    uint64_t lo = s0, hi = s1;  // count of the range's intercepts < x
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        const uint64_t k = sizeof(KT) == 8 ? ld64_hint((const uint64_t*)v.icpt + mid, keep)
                                           : (uint64_t)ld32_hint((const uint32_t*)v.icpt + mid, keep);
        if (k < x) lo = mid + 1;
        else hi = mid;
    }
    if (lo == s0) return k0;  // x <= the first key
    return min(lower_bound_in_segment(v, x, lo - 1, stream), k1);
}

template <typename KT>
__global__ void and_flags_kernel(ColView v, const KT* __restrict__ S, uint64_t nS, uint64_t s0, uint64_t s1, uint64_t k0,
                                 uint64_t k1, uint32_t* __restrict__ flag) {
    const uint64_t keep = policy_keep(), stream = policy_stream();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nS; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = (uint64_t)S[i];
        uint32_t f = 0;
        if (i == 0 || (uint64_t)S[i - 1] != x) {
            const uint64_t p = lower_bound_range<KT>(v, x, s0, s1, k0, k1, keep, stream);
            f = p < k1 && access_one(v, p, keep, stream) == x;
        }
        flag[i] = f;
    }
}

template <typename KT>
__global__ void scatter_flagged_kernel(const KT* __restrict__ S, uint64_t n, const uint32_t* __restrict__ flag,
                                       const uint64_t* __restrict__ off, KT* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        if (flag[i]) out[off[i]] = S[i];
}

constexpr uint32_t kMergeItems = 8;  // merged positions per thread

// Merge path: the number of A elements among the first d of merge(A, B)
// (ties: A first).
template <typename KT>
__device__ __forceinline__ uint64_t merge_split(const KT* A, uint64_t nA, const KT* B, uint64_t nB, uint64_t d) {
    uint64_t lo = d > nB ? d - nB : 0, hi = min(d, nA);
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[d - mid - 1]) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Thread t merges positions [8t, 8t + 8): pass 0 counts the values that
// differ from the merged value before them, pass 1 writes them at off[t].
template <typename KT>
__global__ void or_merge_kernel(const KT* __restrict__ A, uint64_t nA, const KT* __restrict__ B, uint64_t nB, int pass,
                                uint32_t* __restrict__ cnt, const uint64_t* __restrict__ off, KT* __restrict__ out) {
    const uint64_t total = nA + nB, nt = (total + kMergeItems - 1) / kMergeItems;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nt; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d0 = t * kMergeItems, d1 = min(d0 + kMergeItems, total);
        uint64_t i = merge_split(A, nA, B, nB, d0), j = d0 - i;
        bool has_prev = d0 > 0;
        KT prev = 0;
        if (has_prev) {  // merged[d0 - 1]: the larger of the last A and B elements taken
            if (i == 0) prev = B[j - 1];
            else if (j == 0) prev = A[i - 1];
            else prev = max(A[i - 1], B[j - 1]);
        }
        uint64_t o = pass ? off[t] : 0;
        uint32_t c = 0;
        for (uint64_t d = d0; d < d1; ++d) {
            KT x;
            if (j >= nB || (i < nA && A[i] <= B[j])) x = A[i++];
            else x = B[j++];
            if (!has_prev || x != prev) {
                if (pass) out[o++] = x;
                ++c;
            }
            prev = x;
            has_prev = true;
        }
        if (!pass) cnt[t] = c;
    }
}

// ------------------------------------------------------------------ serving: multi-column batches

// Access and lower_bound requests of one batch, over any of the server's
// columns: query q belongs to the last request whose qoff <= q.
template <typename KT>
__global__ void serve_query_kernel(const ColView* __restrict__ views, const SrvReq* __restrict__ reqs, uint32_t nreq,
                                   uint64_t nq, const uint64_t* __restrict__ qin, uint64_t* __restrict__ qout,
                                   uint32_t* __restrict__ status) {
    const uint64_t keep = policy_keep(), stream = policy_stream();
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nq; q += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = nreq - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (reqs[mid].qoff <= q) lo = mid;
            else hi = mid - 1;
        }
        const SrvReq& rq = reqs[lo];
        const ColView& v = views[rq.col];
        const uint64_t x = qin[q];
        if (rq.op == LC_OP_ACCESS) {
            if (x >= v.N) {
                atomicOr(status, kStOutOfRange);
                qout[q] = 0;
            } else {
                qout[q] = access_one(v, x, keep, stream);
            }
        } else {
            qout[q] = lower_bound_one<KT>(v, x, keep, stream);
        }
    }
}

// Range decodes of one batch: work item w is tile first_tile + (w - work_off[r])
// of request r, written to that request's own device buffer.
struct ServeSrc {
    const ColView* views;
    const SrvReq* reqs;
    const uint64_t* work_off;
    uint32_t nreq;
    __device__ void operator()(uint64_t w, const ColView** vv, uint64_t* t, uint64_t* lo, uint64_t* hi,
                               void** o) const {
        const uint64_t a = warp_last_le(work_off, nreq, w);  // the request that holds item w
        const SrvReq& rq = reqs[a];
        *vv = views + rq.col;
        *t = rq.first_tile + (w - work_off[a]);
        *lo = rq.begin;
        *hi = rq.begin + rq.count;
        *o = (void*)rq.out;
    }
};

template <typename KT>
__global__ void __launch_bounds__(kDecThreads, 12)
serve_decode_kernel(const ColView* __restrict__ views, const SrvReq* __restrict__ reqs, uint32_t nreq,
                    const uint64_t* __restrict__ work_off, uint32_t smem_segs) {
    extern __shared__ __align__(16) uint8_t smem[];
    dec_pipeline<KT>(work_off[nreq], ServeSrc{views, reqs, work_off, nreq}, smem, smem_segs);
}

// Derived directories: segment records and rank bits (one CTA per chunk).
template <typename KT>
__global__ void rec_kernel(ColView v, SegRec* __restrict__ recs, RankWord* __restrict__ rank) {
    if (v.gate && *v.gate == 0) return;
    const uint64_t c = blockIdx.x;
    const uint64_t ckb = v.ckb[c], bit0 = 64 * v.cwb[c];
    const uint64_t s1 = v.csb[c + 1];
    const uint32_t nc = (uint32_t)(v.ckb[c + 1] - ckb);
    for (uint64_t j = v.csb[c] + threadIdx.x; j < s1; j += blockDim.x) {
        const uint32_t a = v.start[j];
        const uint32_t e = j + 1 < s1 ? (uint32_t)v.start[j + 1] : nc;
        const uint64_t k = ckb + a;
        SegRec r;
        r.icpt = ld_icpt<KT>(v.icpt, j);
        r.slope = v.slope[j];
        r.kstart_w = k | ((uint64_t)v.width[j] << 56);
        r.bit1_n = (bit0 + v.bitoff[j]) | ((uint64_t)(e - a - 1) << 48);
        recs[j] = r;
        atomicOr((unsigned long long*)&rank[k >> 6].bits, 1ull << (k & 63u));
    }
}

__global__ void rank_pop_kernel(const RankWord* __restrict__ rank, uint64_t nw, uint32_t* __restrict__ pop) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nw; q += (uint64_t)gridDim.x * blockDim.x)
        pop[q] = __popcll(rank[q].bits);
}

__global__ void rank_before_kernel(RankWord* __restrict__ rank, uint64_t nw, const uint64_t* __restrict__ before) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nw; q += (uint64_t)gridDim.x * blockDim.x)
        rank[q].before = before[q];
}

// Radix table: rdx[q] = the number of intercepts < kmin + q 2^shift, i.e.
// the lower bound of the bucket's first value in seg_icpt, for q = 0..nb
// (nb = the buckets [kmin, kmax] spans).  First every 64th entry by a binary
// search over all intercepts, then the others by a binary search between
// their two sampled neighbours (usually a run of a few entries), so that no
// thread's work depends on how the values spread.  The searches stay inside
// [0, L] whatever the intercepts hold (a blob read back from a caller need
// not be sorted).
template <typename KT>
__device__ __forceinline__ uint64_t rdx_lower(const ColView& v, uint64_t q, uint64_t lo, uint64_t hi) {
    if (q > ((~0ull - v.kmin) >> v.rdx_shift)) return hi;  // the bucket starts past 2^64 - 1
    const uint64_t x = v.kmin + (q << v.rdx_shift);
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (ld_icpt<KT>(v.icpt, mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <typename KT>
__global__ void radix_coarse_kernel(ColView v, uint64_t* __restrict__ rdx, uint64_t nb) {
    const uint64_t nc = nb / 64 + 1;  // entries 0, 64, ..., and nb
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c <= nc; c += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = min(64 * c, nb);
        rdx[q] = rdx_lower<KT>(v, q, 0, v.L);
    }
}

template <typename KT>
__global__ void radix_fine_kernel(ColView v, uint64_t* __restrict__ rdx, uint64_t nb) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nb; q += (uint64_t)gridDim.x * blockDim.x) {
        if ((q & 63u) == 0) continue;
        const uint64_t a = q & ~63ull, b = min(a + 64, nb);
        rdx[q] = rdx_lower<KT>(v, q, rdx[a], max(rdx[a], rdx[b]));
    }
}

// ioff[j] = intercept j minus the first value of its radix bucket.
template <typename KT, typename OT>
__global__ void ioff_kernel(ColView v, OT* __restrict__ ioff) {
    const uint64_t mask = (1ull << v.rdx_shift) - 1;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < v.L; j += (uint64_t)gridDim.x * blockDim.x)
        ioff[j] = (OT)((ld_icpt<KT>(v.icpt, j) - v.kmin) & mask);
}

// ends[0] = first key, ends[1] = last key (N >= 1).
__global__ void ends_kernel(ColView v, uint64_t* __restrict__ ends) {
    if (threadIdx.x == 0) {
        ends[0] = v.key_bytes == 4 ? (uint64_t)__ldg((const uint32_t*)v.icpt) : __ldg((const uint64_t*)v.icpt);
        ends[1] = access_one(v, v.N - 1, policy_keep(), policy_stream());
    }
}

__global__ void tile_dir_kernel(ColView v, TileDesc* __restrict__ tiles, uint32_t* __restrict__ max_segs) {
    if (v.gate && *v.gate == 0) return;
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t >= v.ntiles) return;
    uint64_t lo = 0, hi = v.C - 1;  // chunk: last c with chunk_tile_begin[c] <= t
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        if (v.chunk_tile_begin[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const uint64_t c = lo;
    const uint64_t k = t - v.chunk_tile_begin[c];
    const uint64_t ckb = v.ckb[c], nc = v.ckb[c + 1] - ckb;
    const uint32_t local0 = (uint32_t)(k * kTile);
    const uint32_t n = (uint32_t)(nc - local0 < (uint64_t)kTile ? nc - local0 : (uint64_t)kTile);
    const uint32_t local1 = local0 + n - 1;
    auto last_start_le = [&](uint32_t pos) {
        uint64_t a = v.csb[c], b = v.csb[c + 1] - 1;
        while (a < b) {
            const uint64_t mid = (a + b + 1) >> 1;
            if (v.start[mid] <= pos) a = mid;
            else b = mid - 1;
        }
        return a;
    };
    TileDesc d;
    d.key_begin = ckb + local0;
    d.seg_lo = last_start_le(local0);
    d.seg_hi = last_start_le(local1);
    d.chunk = (uint32_t)c;
    d.n = n;
    d.pad = 0;
    // payload words of the residuals of keys local0..local1: from the first
    // residual of seg_lo at or after local0 to the end of seg_hi's residuals up
    // to local1, one word more (an extract reads a word pair), 16-byte aligned
    {
        const uint64_t base = 64 * v.cwb[c];
        const uint32_t s0 = v.start[d.seg_lo], w0 = v.width[d.seg_lo];
        const uint32_t s1 = v.start[d.seg_hi], w1 = v.width[d.seg_hi];
        const uint64_t lo_bit = base + v.bitoff[d.seg_lo] + (uint64_t)w0 * (max(local0, s0 + 1) - s0 - 1);
        const uint64_t hi_bit = base + v.bitoff[d.seg_hi] + (uint64_t)w1 * (local1 - s1);
        const uint64_t wlo = (lo_bit >> 5) & ~3ull;
        uint64_t whi = ((((hi_bit + 31) >> 5) + 1) + 3) & ~3ull;
        if (whi > 2 * v.W) whi = 2 * v.W;
        d.pw0 = wlo;
        d.pwn = hi_bit > lo_bit && whi > wlo ? (uint32_t)(whi - wlo) : 0u;
    }
    tiles[t] = d;
    atomicMax(max_segs, (uint32_t)(d.seg_hi - d.seg_lo + 1));
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <typename KT>
int set_smem() {
    static DeviceOnce once;
    return once_per_device(once, [] {
        cudaError_t e =
            cudaFuncSetAttribute(decode_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDecSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(decode_ranges_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kDecSmem);
        return cuda_status(e);
    });
}

// ------------------------------------------------------------------ partitioned batches of random queries
//
// A large batch of random queries over a column whose directories exceed L2
// misses on each of a query's dependent loads (rank word, record, payload
// word; for lower_bound the radix entry, intercept offsets, record and
// bracket words): about 70 bytes of DRAM each.  Sorted by the part of the
// column they read into buckets of about kPartBucketBytes of directories and
// payload, and run bucket after bucket, the queries of one bucket share an
// L2-resident slice of the column, so each of its lines comes from DRAM about
// once.  The results are the same function of each query; only the order of
// work changes.  The batch is cut into tiles of kPartTile queries, one CTA
// each.  Launches:
//   part_scatter  per tile, a counting sort in shared memory: the tile's
//                 queries in bucket order, written back as one piece at the
//                 tile's place; the start of each bucket's run in the tile;
//                 for each query its position in the sorted tile (16 bits)
//   part_lookup   the runs in bucket-major order (bucket b of every tile,
//                 then bucket b + 1), a warp per run, results written over
//                 the queries
//   part_gather   per tile, its results read back as one piece into shared
//                 memory, then out[q] in query order
// Buckets: key index >> shift for access; for lower_bound the count of
// splitters below the value, the splitters being the keys at multiples of N/B
// (equal key counts per bucket, whatever the value distribution).
constexpr uint32_t kPartThreads = 256;
constexpr uint32_t kPartTile = 4096;                      // queries per tile (CTA)
constexpr uint32_t kPartPer = kPartTile / kPartThreads;   // queries per thread
constexpr uint32_t kPartMaxBuckets = 256;                 // bucket ids fit a byte
constexpr uint64_t kPartBucketBytes = 16ull << 20;
static_assert(kPartMaxBuckets <= kPartThreads, "the tile scan gives one bucket to a thread");
static_assert(kPartTile <= 65536, "positions within a tile are 16-bit");

__device__ __forceinline__ uint64_t policy_normal() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// A coherent streaming load (the lookup writes its results over the keys it read).
__device__ __forceinline__ uint64_t ld_rw_stream(const uint64_t* p, uint64_t pol) {
    uint64_t r;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ void st16_hint(void* ptr, uint16_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u16 [%0], %1, %2;" ::"l"(ptr), "h"(v), "l"(pol) : "memory");
}

struct PartPlan {
    uint32_t B;             // buckets, <= kPartMaxBuckets
    uint32_t dense;         // 1: the lookups read a decoded copy of the column
    uint32_t shift;         // access: bucket = index >> shift
    const uint64_t* split;  // lower_bound: B - 1 ascending keys
    uint64_t T;             // tiles
    uint64_t N;
};

template <bool BY_VALUE>
__device__ __forceinline__ uint32_t part_bucket(uint64_t key, const PartPlan& pp, const uint64_t* s_split) {
    if (!BY_VALUE) return (uint32_t)((key < pp.N ? key : pp.N - 1) >> pp.shift);
    uint32_t lo = 0, hi = pp.B - 1;  // count of splitters < key
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_split[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <bool BY_VALUE>
__device__ __forceinline__ void part_load_split(const PartPlan& pp, uint64_t* s_split) {
    if (BY_VALUE)
        for (uint32_t k = threadIdx.x; k + 1 < pp.B; k += blockDim.x) s_split[k] = pp.split[k];
}

// Exclusive prefix sum of s[0, B) in place (B <= blockDim.x = kPartThreads).
__device__ __forceinline__ void tile_scan(uint32_t* s, uint32_t B, uint32_t* s_warp) {
    const uint32_t t = threadIdx.x, lane = t & 31u, w = t >> 5;
    const uint32_t v = t < B ? s[t] : 0u;
    uint32_t x = v;
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(~0u, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t z = lane < kPartThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (uint32_t d = 1; d < kPartThreads / 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(~0u, z, d);
            if (lane >= d) z += y;
        }
        if (lane < kPartThreads / 32) s_warp[lane] = z;
    }
    __syncthreads();
    if (t < B) s[t] = (w ? s_warp[w - 1] : 0u) + x - v;
    __syncthreads();
}

// Splitters for lower_bound: the key at floor((k + 1) N / B), k < B - 1.
__global__ void part_split_kernel(ColView v, uint32_t B, uint64_t* __restrict__ split) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k + 1 >= B) return;
    const uint64_t q = v.N / B, r = v.N % B;
    const uint64_t i = q * (k + 1) + r * (k + 1) / B;  // r (k + 1) < B^2
    split[k] = access_one(v, i, policy_keep(), policy_normal());
}

template <bool BY_VALUE, typename QT>
__global__ void __launch_bounds__(kPartThreads) part_scatter_kernel(const QT* __restrict__ keys, uint64_t m, PartPlan pp,
                                                                    uint64_t* __restrict__ bkey,
                                                                    uint16_t* __restrict__ runs,
                                                                    uint16_t* __restrict__ pos) {
    __shared__ uint64_t s_key[kPartTile];  // the tile's queries in bucket order
    __shared__ uint32_t s_cnt[kPartMaxBuckets];
    __shared__ uint64_t s_split[BY_VALUE ? kPartMaxBuckets : 1];
    __shared__ uint32_t s_warp[kPartThreads / 32];
    const uint64_t c = blockIdx.x, q0 = c * kPartTile;
    const uint32_t nt = (uint32_t)min((uint64_t)kPartTile, m - q0);
    for (uint32_t b = threadIdx.x; b < pp.B; b += blockDim.x) s_cnt[b] = 0;
    part_load_split<BY_VALUE>(pp, s_split);
    __syncthreads();
    const uint64_t pol = policy_stream();
    uint64_t kk[kPartPer];
    uint32_t code[kPartPer];  // bucket << 16 | rank within the bucket
#pragma unroll
    for (uint32_t u = 0; u < kPartPer; ++u) {
        const uint32_t j = u * kPartThreads + threadIdx.x;
        kk[u] = j < nt ? ld_stream(keys + q0 + j, pol) : 0;
    }
#pragma unroll
    for (uint32_t u = 0; u < kPartPer; ++u) {
        if (u * kPartThreads + threadIdx.x < nt) {
            const uint32_t b = part_bucket<BY_VALUE>(kk[u], pp, s_split);
            code[u] = (b << 16) | atomicAdd(&s_cnt[b], 1u);
        }
    }
    __syncthreads();
    tile_scan(s_cnt, pp.B, s_warp);  // s_cnt[b]: first position of bucket b in the sorted tile
#pragma unroll
    for (uint32_t u = 0; u < kPartPer; ++u) {
        const uint32_t j = u * kPartThreads + threadIdx.x;
        if (j < nt) {
            const uint32_t at = s_cnt[code[u] >> 16] + (code[u] & 0xffffu);
            s_key[at] = kk[u];
            st16_hint(pos + q0 + j, (uint16_t)at, pol);
        }
    }
    uint16_t* rc = runs + c * (pp.B + 1);
    for (uint32_t b = threadIdx.x; b <= pp.B; b += blockDim.x) rc[b] = (uint16_t)(b < pp.B ? s_cnt[b] : nt);
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nt; j += kPartThreads) bkey[q0 + j] = s_key[j];
}

// The first index in [ks + 1, ks + n] whose decoded key is >= x, given that
// the key at ks (segment j's intercept) is < x: a binary search of the decoded
// keys of the segment.
template <typename KT>
__device__ __forceinline__ uint64_t lower_bound_decoded(const ColView& v, const KT* __restrict__ D, uint64_t x,
                                                        uint64_t pol) {
    if (v.L == 0 || x <= v.kmin) return 0;
    if (x > v.kmax) return v.N;
    const SegRec r = load_rec_hint(v.recs + segment_below<KT>(v, x, pol), pol);
    const uint64_t ks = r.kstart_w & kKeyMask;
    uint32_t a = 1, b = (uint32_t)(r.bit1_n >> 48) + 1u;
    while (a < b) {
        const uint32_t mid = (a + b) >> 1;
        const uint64_t k = sizeof(KT) == 8 ? ld64_hint(D + ks + mid, pol) : (uint64_t)ld32_hint(D + ks + mid, pol);
        if (k < x) a = mid + 1;
        else b = mid;
    }
    return ks + a;
}

// The runs in bucket-major order (bucket b of every tile, then bucket b + 1),
// a warp per run, grid-stride over the runs: the runs in flight at once are
// consecutive, so they keep to one bucket or two (two queries per lane, or
// four runs per warp, measured slower), and the next run's bounds are loaded
// while this one's queries run.  The column's lines are read with the normal
// L2 priority: a bucket's slice is reused by its queries, the query stream is
// not.  DENSE: D holds every key decoded; access reads its key there,
// lower_bound searches there inside the segment the directories give.
template <bool BY_VALUE, bool DENSE, typename KT>
__device__ __forceinline__ uint64_t part_answer(const ColView& v, const KT* __restrict__ D, uint64_t key,
                                                uint64_t normal) {
    if (BY_VALUE)
        return DENSE ? lower_bound_decoded<KT>(v, D, key, normal) : lower_bound_one<KT>(v, key, normal, normal);
    if (key < v.N)
        return DENSE ? (sizeof(KT) == 8 ? ld64_hint(D + key, normal) : (uint64_t)ld32_hint(D + key, normal))
                     : access_one(v, key, normal, normal);
    atomicOr(v.status, kStOutOfRange);
    return 0;
}

template <bool BY_VALUE, bool DENSE, typename KT>
__global__ void __launch_bounds__(256, 6) part_lookup_kernel(ColView v, const KT* __restrict__ D,
                                                             uint64_t* __restrict__ bkey,
                                                             const uint16_t* __restrict__ runs, PartPlan pp) {
    const uint64_t normal = policy_normal(), stream = policy_stream();
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t nruns = (uint64_t)pp.B * pp.T;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    // run r: bucket r / T of tile r % T; its queries' slots [c kPartTile + s, c kPartTile + e)
    auto bounds = [&](uint64_t r, uint64_t& first, uint32_t& len) {
        const uint64_t b = r / pp.T, c = r - b * pp.T;
        const uint16_t* rc = runs + c * (pp.B + 1) + b;
        const uint32_t s0 = __ldg(rc), e0 = __ldg(rc + 1);
        first = c * kPartTile + s0;
        len = e0 - s0;
    };
    uint64_t r = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    if constexpr (DENSE && !BY_VALUE) {
        // One load per answer: the first 64 queries of the next run, and the
        // bounds of the one after, are loaded while this run's keys are read,
        // so that a run costs about one memory latency rather than two per
        // 32 queries.  A run's stores and the next run's loads touch disjoint
        // slots.
        if (r >= nruns) return;
        uint64_t f0, f1 = 0;
        uint32_t l0, l1 = 0;
        bounds(r, f0, l0);
        uint64_t qa = lane < l0 ? ld_rw_stream(bkey + f0 + lane, stream) : 0;
        uint64_t qb = lane + 32 < l0 ? ld_rw_stream(bkey + f0 + lane + 32, stream) : 0;
        if (r + warps < nruns) bounds(r + warps, f1, l1);
        for (;;) {
            const uint64_t ra = lane < l0 ? part_answer<false, true, KT>(v, D, qa, normal) : 0;
            const uint64_t rb = lane + 32 < l0 ? part_answer<false, true, KT>(v, D, qb, normal) : 0;
            const bool more = r + warps < nruns;
            uint64_t na = 0, nb = 0, f2 = 0;
            uint32_t l2 = 0;
            if (more) {
                na = lane < l1 ? ld_rw_stream(bkey + f1 + lane, stream) : 0;
                nb = lane + 32 < l1 ? ld_rw_stream(bkey + f1 + lane + 32, stream) : 0;
                if (r + 2 * warps < nruns) bounds(r + 2 * warps, f2, l2);
            }
            for (uint32_t k = 64 + lane; k < l0; k += 32)  // the rest of a long run
                st64_hint(bkey + f0 + k, part_answer<false, true, KT>(v, D, ld_rw_stream(bkey + f0 + k, stream), normal),
                          stream);
            if (lane < l0) st64_hint(bkey + f0 + lane, ra, stream);
            if (lane + 32 < l0) st64_hint(bkey + f0 + lane + 32, rb, stream);
            if (!more) return;
            r += warps;
            f0 = f1, l0 = l1, qa = na, qb = nb, f1 = f2, l1 = l2;
        }
    }
    uint64_t nfirst = 0;
    uint32_t nlen = 0;
    if (r < nruns) bounds(r, nfirst, nlen);
    for (; r < nruns; r += warps) {
        const uint64_t first = nfirst;
        const uint32_t len = nlen;
        if (r + warps < nruns) bounds(r + warps, nfirst, nlen);
        for (uint32_t k = lane; k < len; k += 32)
            st64_hint(bkey + first + k,
                      part_answer<BY_VALUE, DENSE, KT>(v, D, ld_rw_stream(bkey + first + k, stream), normal), stream);
    }
}

template <typename OT>
__global__ void __launch_bounds__(kPartThreads) part_gather_kernel(const uint64_t* __restrict__ res,
                                                                   const uint16_t* __restrict__ pos, uint64_t m,
                                                                   OT* __restrict__ out) {
    __shared__ uint64_t s_res[kPartTile];  // the tile's results in bucket order
    const uint64_t c = blockIdx.x, q0 = c * kPartTile;
    const uint32_t nt = (uint32_t)min((uint64_t)kPartTile, m - q0);
    const uint64_t stream = policy_stream();
    uint32_t pq[kPartPer];  // each query's position in the sorted tile, loaded early
#pragma unroll
    for (uint32_t u = 0; u < kPartPer; ++u) {
        const uint32_t j = u * kPartThreads + threadIdx.x;
        pq[u] = j < nt ? (uint32_t)ld_stream(pos + q0 + j, stream) : 0u;
    }
#pragma unroll
    for (uint32_t u = 0; u < kPartPer; ++u) {
        const uint32_t j = u * kPartThreads + threadIdx.x;
        if (j < nt) s_res[j] = ld_stream(res + q0 + j, stream);
    }
    __syncthreads();
#pragma unroll
    for (uint32_t u = 0; u < kPartPer; ++u) {
        const uint32_t j = u * kPartThreads + threadIdx.x;
        if (j < nt) st_stream(out + q0 + j, s_res[pq[u]], stream);
    }
}

}  // namespace

Derived2Layout derived2_layout(uint64_t N, uint64_t L, bool list_mode) {
    Derived2Layout d;
    // (lower_bound needs sorted keys: no table in list mode)
    uint32_t blog = 0;  // B = 2^blog buckets, about two per segment, at most 2^kRdxMaxLog
    while (blog < kRdxMaxLog && (1ull << blog) < 2 * L) ++blog;
    d.B = list_mode ? 0 : 1ull << blog;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    d.off_rank = al(sizeof(SegRec) * L);
    d.off_rdx = al(d.off_rank + sizeof(RankWord) * ((N + 63) / 64));
    d.off_ioff = al(d.off_rdx + (d.B ? 8 * (d.B + 1) : 0));
    d.bytes = al(d.off_ioff + (d.B ? 4 * L : 0)) + 256;
    return d;
}

int build_derived(lc_column* col, cudaStream_t st) {
    const uint64_t C = col->C, L = col->L, N = col->N;
    // the segment records hold key indices in 56 bits and payload bits in 48
    if (N >= (1ull << 56) || col->W >= (1ull << 42)) return LC_ERR_UNSUPPORTED;
    // host: tiles per chunk from the chunk directory
    std::vector<uint64_t> ctb(C + 1, 0);
    for (uint64_t c = 0; c < C; ++c) {
        const uint64_t nc = col->h_ckb[c + 1] - col->h_ckb[c];
        ctb[c + 1] = ctb[c] + (nc + kTile - 1) / kTile;
    }
    col->ntiles = ctb[C];
    col->h_ctb = new (std::nothrow) uint64_t[C + 1];
    if (!col->h_ctb) return LC_ERR_NOMEM;
    std::copy(ctb.begin(), ctb.end(), col->h_ctb);
    const size_t bytes = 8 * (C + 1) + sizeof(TileDesc) * (col->ntiles + 1) + 256;
    uint8_t* p = nullptr;
    if (cudaMallocAsync((void**)&p, bytes, st) != cudaSuccess) return LC_ERR_NOMEM;
    col->chunk_tile_begin = (uint64_t*)p;
    col->tiles = (TileDesc*)(p + 8 * (C + 1));
    col->status = (uint32_t*)(p + 8 * (C + 1) + sizeof(TileDesc) * (col->ntiles + 1));
    int rc = stage_h2d(col->chunk_tile_begin, ctb.data(), 8 * (C + 1), st);
    if (rc) return rc;
    rc = cuda_status(cudaMemsetAsync(col->status, 0, 4, st));
    if (rc) return rc;

    // segment records, rank words, the radix table over the intercepts (the
    // memory may have been taken while the compress's last stage ran)
    const uint64_t nw = (N + 63) / 64;
    const Derived2Layout dl = derived2_layout(N, L, col->list_mode != 0);
    const uint64_t B = dl.B;
    const size_t off_rank = dl.off_rank, off_rdx = dl.off_rdx, off_ioff = dl.off_ioff;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    if (!col->derived2 && cudaMallocAsync((void**)&col->derived2, dl.bytes, st) != cudaSuccess) {
        col->derived2 = nullptr;
        return LC_ERR_NOMEM;
    }
    if ((uintptr_t)col->derived2 % 32) return LC_ERR_INTERNAL;  // records are read with 32-byte loads
    SegRec* recs = (SegRec*)col->derived2;
    RankWord* rank = (RankWord*)(col->derived2 + off_rank);
    uint64_t* rdx = (uint64_t*)(col->derived2 + off_rdx);
    if (nw) {
        rc = cuda_status(cudaMemsetAsync(rank, 0, sizeof(RankWord) * nw, st));
        if (rc) return rc;
    }

    ColView& v = col->view;
    const Layout& Ly = col->lay;
    v.ckb = (const uint64_t*)(col->blob + Ly.ckb);
    v.csb = (const uint64_t*)(col->blob + Ly.csb);
    v.cwb = (const uint64_t*)(col->blob + Ly.cwb);
    v.icpt = col->blob + Ly.icpt;
    v.slope = (const int64_t*)(col->blob + Ly.slope);
    v.bitoff = (const uint32_t*)(col->blob + Ly.bitoff);
    v.start = (const uint16_t*)(col->blob + Ly.start);
    v.width = (const uint8_t*)(col->blob + Ly.width);
    v.pay32 = (const uint32_t*)(col->blob + Ly.payload);
    v.tiles = col->tiles;
    v.chunk_tile_begin = col->chunk_tile_begin;
    v.recs = recs;
    v.rank = rank;
    v.rdx = B ? rdx : nullptr;
    v.ioff = nullptr;
    v.ioff_bytes = 0;
    v.kmin = v.kmax = 0;
    v.rdx_shift = 0;
    v.key_bytes = col->key_bytes;
    v.status = col->status;
    v.gate = nullptr;
    v.N = N;
    v.C = C;
    v.L = L;
    v.W = col->W;
    v.ntiles = col->ntiles;
    v.chunk_log2 = col->chunk_log2;
    v.list_mode = col->list_mode;
    if (C) {
        rc = cuda_status(cudaMemsetAsync(col->status + 1, 0, 4, st));
        if (rc) return rc;
        {
            KTime kt("derived", st);
            tile_dir_kernel<<<(unsigned)((col->ntiles + 255) / 256), 256, 0, st>>>(v, col->tiles, col->status + 1);
            if (col->key_bytes == 4) rec_kernel<uint32_t><<<(unsigned)C, 128, 0, st>>>(v, recs, rank);
            else rec_kernel<uint64_t><<<(unsigned)C, 128, 0, st>>>(v, recs, rank);
        }
        note_launch(2);
        rc = cuda_status(cudaGetLastError());
        if (rc) return rc;
        // rank prefix: popcounts, exclusive scan, scatter
        const size_t tmpb = scan_tmp_bytes(nw);
        uint8_t* t = nullptr;
        if (cudaMallocAsync((void**)&t, al(4 * nw) + al(8 * (nw + 1)) + tmpb, st) != cudaSuccess) return LC_ERR_NOMEM;
        uint32_t* pop = (uint32_t*)t;
        uint64_t* before = (uint64_t*)(t + al(4 * nw));
        const unsigned g = (unsigned)std::min<uint64_t>((nw + 255) / 256, 65535);
        rank_pop_kernel<<<g, 256, 0, st>>>(rank, nw, pop);
        note_launch();
        rc = scan_exclusive(pop, before, nw, ScanOp::Identity, t + al(4 * nw) + al(8 * (nw + 1)), tmpb, st);
        if (!rc) {
            rank_before_kernel<<<g, 256, 0, st>>>(rank, nw, before);
            note_launch();
            rc = cuda_status(cudaGetLastError());
        }
        cudaFreeAsync(t, st);
        if (rc) return rc;
        // first and last key, and the most segments one decode tile meets
        uint64_t* ends = (uint64_t*)(col->status + 2);
        ends_kernel<<<1, 32, 0, st>>>(v, ends);
        note_launch();
        uint64_t h[3] = {0, 0, 0};
        const void* ph = nullptr;
        rc = stage_d2h(col->status, 24, st, &ph);
        if (rc) return rc;
        rc = stage_sync(st);
        if (rc) return rc;
        std::memcpy(h, ph, 24);
        v.max_tile_segs = std::max<uint32_t>((uint32_t)(h[0] >> 32), 1);
        v.kmin = h[1];
        v.kmax = h[2];
        if (!B) return LC_OK;
        uint32_t sh = 0;
        while (sh < 64 && ((v.kmax - v.kmin) >> sh) >= B) ++sh;
        v.rdx_shift = sh;
        const uint64_t nb = v.kmax >= v.kmin ? ((v.kmax - v.kmin) >> sh) + 1 : 1;  // buckets in use, <= B
        {
            KTime kt("derived_radix", st);
            const unsigned gc = (unsigned)std::min<uint64_t>((nb / 64 + 2 + 255) / 256, 65535);
            const unsigned gf = (unsigned)std::min<uint64_t>((nb + 255) / 256, 65535);
            if (col->key_bytes == 4) {
                radix_coarse_kernel<uint32_t><<<gc, 256, 0, st>>>(v, rdx, nb);
                radix_fine_kernel<uint32_t><<<gf, 256, 0, st>>>(v, rdx, nb);
            } else {
                radix_coarse_kernel<uint64_t><<<gc, 256, 0, st>>>(v, rdx, nb);
                radix_fine_kernel<uint64_t><<<gf, 256, 0, st>>>(v, rdx, nb);
            }
        }
        note_launch(2);
        rc = cuda_status(cudaGetLastError());
        if (rc) return rc;
        // intercept offsets within their buckets, 16 or 32 bits when the buckets are that narrow
        if (sh <= 32) {
            uint8_t* ioff = col->derived2 + off_ioff;
            const unsigned gi = (unsigned)std::min<uint64_t>((L + 255) / 256, 65535);
            KTime kt("derived_radix", st);
            if (sh <= 16) {
                if (col->key_bytes == 4) ioff_kernel<uint32_t, uint16_t><<<gi, 256, 0, st>>>(v, (uint16_t*)ioff);
                else ioff_kernel<uint64_t, uint16_t><<<gi, 256, 0, st>>>(v, (uint16_t*)ioff);
            } else {
                if (col->key_bytes == 4) ioff_kernel<uint32_t, uint32_t><<<gi, 256, 0, st>>>(v, (uint32_t*)ioff);
                else ioff_kernel<uint64_t, uint32_t><<<gi, 256, 0, st>>>(v, (uint32_t*)ioff);
            }
            note_launch();
            rc = cuda_status(cudaGetLastError());
            if (rc) return rc;
            v.ioff = ioff;
            v.ioff_bytes = sh <= 16 ? 2 : 4;
        }
        return cuda_status(cudaStreamSynchronize(st));
    }
    v.max_tile_segs = 1;
    return cuda_status(cudaStreamSynchronize(st));
}

// Host-side tile index of key i (uses the host copies of the directories).
static uint64_t host_tile_of(const lc_column* col, uint64_t i) {
    uint64_t c;
    if (!col->list_mode) {
        c = i >> col->chunk_log2;
    } else {
        c = (uint64_t)(std::upper_bound(col->h_ckb, col->h_ckb + col->C + 1, i) - col->h_ckb) - 1;
    }
    return col->h_ctb[c] + ((i - col->h_ckb[c]) >> kTileLog);
}

// CTAs of a persistent decode launch: as many as fit on every SM at once.
template <typename F>
static unsigned dec_grid(F kernel, size_t smem) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kDecThreads, smem) != cudaSuccess || occ < 1)
        occ = 1;
    return (unsigned)(sm_count() * occ);
}

template <typename KT>
static int launch_decode(const lc_column* col, uint64_t t0, uint64_t nt, uint64_t begin, uint64_t count, void* out,
                         cudaStream_t st, const ColView* view = nullptr, const char* name = "decode") {
    int rc = set_smem<KT>();
    if (rc) return rc;
    const ColView& v = view ? *view : col->view;
    const size_t smem = dec_smem(v.max_tile_segs);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decode_kernel<KT>, kDecThreads, smem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    const uint64_t grid = std::min<uint64_t>(nt, (uint64_t)sm_count() * occ);
    {
        KTime kt(name, st);
        decode_kernel<KT><<<(unsigned)grid, kDecThreads, smem, st>>>(v, t0, nt, begin, begin + count, (KT*)out);
    }
    note_launch();
    return cuda_status(cudaGetLastError());
}

int decode_range(const lc_column* col, uint64_t begin, uint64_t count, void* out, cudaStream_t st) {
    if (count == 0) return LC_OK;
    const uint64_t t0 = host_tile_of(col, begin), t1 = host_tile_of(col, begin + count - 1);
    if (col->key_bytes == 4) return launch_decode<uint32_t>(col, t0, t1 - t0 + 1, begin, count, out, st);
    return launch_decode<uint64_t>(col, t0, t1 - t0 + 1, begin, count, out, st);
}

size_t derived_replay_tmp_bytes(const lc_column* col) {
    const uint64_t nw = (col->N + 63) / 64;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return al(4 * nw) + al(8 * (nw + 1)) + scan_tmp_bytes(nw);
}

int derived_replay(lc_column* col, const uint32_t* gate, void* tmp, size_t tmp_bytes, void* out, cudaStream_t st) {
    if (!col->list_mode || col->C == 0) return LC_ERR_INVALID_ARG;
    if (tmp_bytes < derived_replay_tmp_bytes(col)) return LC_ERR_INTERNAL;
    ColView v = col->view;
    v.gate = gate;
    const uint64_t nw = (col->N + 63) / 64;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    RankWord* rank = const_cast<RankWord*>(v.rank);
    int rc = cuda_status(cudaMemsetAsync(rank, 0, sizeof(RankWord) * nw, st));
    if (rc) return rc;
    tile_dir_kernel<<<(unsigned)((col->ntiles + 255) / 256), 256, 0, st>>>(v, col->tiles, col->status + 1);
    if (col->key_bytes == 4) rec_kernel<uint32_t><<<(unsigned)col->C, 128, 0, st>>>(v, const_cast<SegRec*>(v.recs), rank);
    else rec_kernel<uint64_t><<<(unsigned)col->C, 128, 0, st>>>(v, const_cast<SegRec*>(v.recs), rank);
    note_launch(2);
    rc = cuda_status(cudaGetLastError());
    if (rc) return rc;
    uint8_t* t = (uint8_t*)tmp;
    uint32_t* pop = (uint32_t*)t;
    uint64_t* before = (uint64_t*)(t + al(4 * nw));
    const unsigned g = (unsigned)std::min<uint64_t>((nw + 255) / 256, 65535);
    rank_pop_kernel<<<g, 256, 0, st>>>(rank, nw, pop);
    note_launch();
    rc = scan_exclusive(pop, before, nw, ScanOp::Identity, t + al(4 * nw) + al(8 * (nw + 1)), scan_tmp_bytes(nw), st);
    if (rc) return rc;
    rank_before_kernel<<<g, 256, 0, st>>>(rank, nw, before);
    note_launch();
    rc = cuda_status(cudaGetLastError());
    if (rc || !out) return rc;
    const uint64_t nt = col->ntiles;
    if (col->key_bytes == 4) return launch_decode<uint32_t>(col, 0, nt, 0, col->N, out, st, &v);
    return launch_decode<uint64_t>(col, 0, nt, 0, col->N, out, st, &v);
}

int decode_ranges(const lc_column* col, const uint64_t* begin, const uint64_t* count, const uint64_t* out_off,
                  uint64_t m, void* out, uint64_t out_cap, cudaStream_t st) {
    if (m == 0) return LC_OK;
    const size_t tmp_b = scan_tmp_bytes(m);
    const size_t bytes = 8 * m + 4 * m + 8 * (m + 1) + tmp_b + 64;
    uint8_t* p = nullptr;
    if (cudaMallocAsync((void**)&p, bytes, st) != cudaSuccess) return LC_ERR_NOMEM;
    uint64_t* first = (uint64_t*)p;
    uint64_t* work_off = first + m;
    uint32_t* ntiles = (uint32_t*)(work_off + m + 1);
    void* tmp = (void*)(((uintptr_t)(ntiles + m) + 15) & ~(uintptr_t)15);
    range_tiles_kernel<<<(unsigned)std::min<uint64_t>((m + 255) / 256, 4096), 256, 0, st>>>(
        col->view, begin, count, out_off, out_cap, m, first, ntiles);
    note_launch();
    int rc = cuda_status(cudaGetLastError());
    if (!rc) rc = scan_exclusive(ntiles, work_off, m, ScanOp::Identity, tmp, tmp_b, st);
    if (!rc) {
        const size_t smem = dec_smem(col->view.max_tile_segs);
        if (col->key_bytes == 4) {
            if (!(rc = set_smem<uint32_t>())) {
                const unsigned grid = dec_grid(decode_ranges_kernel<uint32_t>, smem);
                KTime kt("decode_ranges", st);
                decode_ranges_kernel<uint32_t><<<grid, kDecThreads, smem, st>>>(col->view, begin, count, out_off, m,
                                                                               first, work_off, (uint32_t*)out);
            }
        } else {
            if (!(rc = set_smem<uint64_t>())) {
                const unsigned grid = dec_grid(decode_ranges_kernel<uint64_t>, smem);
                KTime kt("decode_ranges", st);
                decode_ranges_kernel<uint64_t><<<grid, kDecThreads, smem, st>>>(col->view, begin, count, out_off, m,
                                                                               first, work_off, (uint64_t*)out);
            }
        }
        if (!rc) {
            note_launch();
            rc = cuda_status(cudaGetLastError());
        }
    }
    cudaFreeAsync(p, st);
    return rc;
}

// How a batch of access / lower_bound queries runs (lc_set_query_plan).
static std::atomic<int> g_query_plan{LC_QUERIES_AUTO};

int set_query_plan(int plan) {
    if (plan != LC_QUERIES_AUTO && plan != LC_QUERIES_DIRECT && plan != LC_QUERIES_PARTITIONED &&
        plan != LC_QUERIES_DECODED)
        return LC_ERR_INVALID_ARG;
    return g_query_plan.exchange(plan);
}

namespace {

constexpr uint64_t kPartMinQueries = 1ull << 21;
constexpr uint64_t kPartMinDirBytes = 96ull << 20;  // about three quarters of L2
constexpr uint64_t kPartMinDecodedBytes = 64ull << 20;

// The bucket plan of a batch of m queries, or false when the batch runs
// direct.  Under LC_QUERIES_AUTO:
// * a dense access batch (at least one query per 8 keys) on a column whose
//   keys take 64 MB or more runs decoded: one bulk decode of the column, then
//   each query reads its key from the decoded copy, bucket by bucket;
// * else an access batch runs partitioned through the directories when it is
//   large, the records and rank words exceed three quarters of L2, and there
//   is at least one query per 32 bytes of directories and payload -- then a
//   direct lookup would miss L2 on each dependent load, while the partitioned
//   lookup is bound by the L2's request rate;
// * else direct.  A lower_bound batch always runs direct: its lookup is bound
//   by instruction issue (the search inside the segment) more than by DRAM,
//   and a search of the decoded keys is a chain of dependent loads.
bool part_plan(const lc_column* col, uint64_t m, bool by_value, PartPlan* pp) {
    const int plan = g_query_plan.load(std::memory_order_relaxed);
    const ColView& v = col->view;
    if (plan == LC_QUERIES_DIRECT || m >= (1ull << 32) || v.N == 0) return false;
    const uint64_t kb = col->key_bytes;
    const uint64_t dir = by_value ? 32 * v.L + 8 * (((v.kmax - v.kmin) >> v.rdx_shift) + 2) + (uint64_t)v.ioff_bytes * v.L
                                  : 32 * v.L + 16 * ((v.N + 63) / 64);
    bool dense;
    if (plan == LC_QUERIES_AUTO) {
        const bool big = m >= kPartMinQueries;
        if (by_value) return false;
        dense = big && 8 * m >= v.N && kb * v.N >= kPartMinDecodedBytes;
        if (!dense && (!big || dir < kPartMinDirBytes || 32 * m < dir + 8 * v.W)) return false;
    } else {
        dense = plan == LC_QUERIES_DECODED;
    }
    // bytes a bucket's lookups read: the decoded keys (and for lower_bound the
    // directories), or the directories and the payload
    const uint64_t bytes = dense ? kb * v.N + (by_value ? dir : 0) : dir + 8 * v.W;
    uint64_t B = (bytes + kPartBucketBytes - 1) / kPartBucketBytes;
    if (plan != LC_QUERIES_AUTO) B = std::max<uint64_t>(B, 16);  // several buckets even on small columns
    B = std::min<uint64_t>(std::max<uint64_t>(B, 1), kPartMaxBuckets);
    pp->dense = dense ? 1u : 0u;
    pp->N = v.N;
    pp->split = nullptr;
    pp->shift = 0;
    if (!by_value) {  // buckets of 2^shift key indices
        const uint64_t per = (v.N + B - 1) / B;
        while ((1ull << pp->shift) < per) ++pp->shift;
        pp->B = (uint32_t)(((v.N - 1) >> pp->shift) + 1);
    } else {
        pp->B = (uint32_t)B;
    }
    pp->T = (m + kPartTile - 1) / kPartTile;
    return true;
}

// A partitioned batch: keys are the m indices (access) or values
// (lower_bound), out the m results.  Scratch from the stream-ordered pool,
// released in stream order: 10 bytes per query plus 2 per bucket and tile,
// and the decoded column when the plan is dense.
template <bool BY_VALUE, typename KT, typename QT, typename OT>
int run_partitioned(const lc_column* col, const QT* keys, uint64_t m, PartPlan pp, OT* out, cudaStream_t st) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_pos = al(8 * m), o_runs = o_pos + al(2 * m), o_split = o_runs + al(2 * pp.T * (pp.B + 1));
    const size_t o_dec = o_split + al(8 * pp.B);
    const size_t total = o_dec + (pp.dense ? al(sizeof(KT) * col->N) : 0);
    uint8_t* p = nullptr;
    if (cudaMallocAsync((void**)&p, total, st) != cudaSuccess) return LC_ERR_NOMEM;
    uint64_t* bkey = (uint64_t*)p;
    uint16_t* pos = (uint16_t*)(p + o_pos);
    uint16_t* runs = (uint16_t*)(p + o_runs);
    uint64_t* split = (uint64_t*)(p + o_split);
    KT* dec = pp.dense ? (KT*)(p + o_dec) : nullptr;
    int rc = LC_OK;
    if (pp.dense)  // every key, decoded once (the bulk decode launch)
        rc = launch_decode<KT>(col, 0, col->ntiles, 0, col->N, dec, st, nullptr,
                               BY_VALUE ? "lower_bound.decode" : "access.decode");
    if (BY_VALUE && !rc) {
        pp.split = split;
        if (pp.B > 1) {
            part_split_kernel<<<(pp.B + 255) / 256, 256, 0, st>>>(col->view, pp.B, split);
            note_launch();
            rc = cuda_status(cudaGetLastError());
        }
    }
    if (!rc) {
        KTime kt(BY_VALUE ? "lower_bound.scatter" : "access.scatter", st);
        part_scatter_kernel<BY_VALUE, QT><<<(unsigned)pp.T, kPartThreads, 0, st>>>(keys, m, pp, bkey, runs, pos);
        note_launch();
        rc = cuda_status(cudaGetLastError());
    }
    if (!rc) {
        auto kern = pp.dense ? part_lookup_kernel<BY_VALUE, true, KT> : part_lookup_kernel<BY_VALUE, false, KT>;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0) != cudaSuccess || occ < 1) occ = 1;
        const uint64_t nruns = (uint64_t)pp.B * pp.T;  // a warp per run
        const unsigned grid = (unsigned)std::min<uint64_t>((nruns + 7) / 8, (uint64_t)sm_count() * occ);
        KTime kt(BY_VALUE ? "lower_bound.lookup" : "access.lookup", st);
        kern<<<grid, 256, 0, st>>>(col->view, dec, bkey, runs, pp);
        note_launch();
        rc = cuda_status(cudaGetLastError());
    }
    if (!rc) {
        KTime kt(BY_VALUE ? "lower_bound.gather" : "access.gather", st);
        part_gather_kernel<OT><<<(unsigned)pp.T, kPartThreads, 0, st>>>(bkey, pos, m, out);
        note_launch();
        rc = cuda_status(cudaGetLastError());
    }
    const int rf = cuda_status(cudaFreeAsync(p, st));
    return rc ? rc : rf;
}

}  // namespace

int access(const lc_column* col, const uint64_t* idx, uint64_t m, void* out, cudaStream_t st) {
    if (m == 0) return LC_OK;
    PartPlan pp;
    if (part_plan(col, m, false, &pp)) {
        KTime kt("access", st);
        if (col->key_bytes == 4)
            return run_partitioned<false, uint32_t>(col, idx, m, pp, (uint32_t*)out, st);
        return run_partitioned<false, uint64_t>(col, idx, m, pp, (uint64_t*)out, st);
    }
    const unsigned grid = (unsigned)std::min<uint64_t>((m + 255) / 256, (uint64_t)sm_count() * 16);
    {
        KTime kt("access", st);
        if (col->key_bytes == 4) access_kernel<uint32_t><<<grid, 256, 0, st>>>(col->view, idx, m, (uint32_t*)out);
        else access_kernel<uint64_t><<<grid, 256, 0, st>>>(col->view, idx, m, (uint64_t*)out);
    }
    note_launch();
    return cuda_status(cudaGetLastError());
}

int lower_bound(const lc_column* col, const void* vals, uint64_t m, uint64_t* out, cudaStream_t st) {
    if (m == 0) return LC_OK;
    const ColView& v = col->view;
    PartPlan pp;
    if (part_plan(col, m, true, &pp)) {
        KTime kt("lower_bound", st);
        if (col->key_bytes == 4)
            return run_partitioned<true, uint32_t>(col, (const uint32_t*)vals, m, pp, out, st);
        return run_partitioned<true, uint64_t>(col, (const uint64_t*)vals, m, pp, out, st);
    }
    // one query per thread, as many CTAs as stay resident (grid-stride)
    int occ = 0;
    const cudaError_t oe = col->key_bytes == 4
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lower_bound_kernel<uint32_t>, 256, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lower_bound_kernel<uint64_t>, 256, 0);
    if (oe != cudaSuccess || occ < 1) occ = 1;
    const unsigned grid = (unsigned)std::min<uint64_t>((m + 255) / 256, (uint64_t)sm_count() * occ);
    {
        KTime kt("lower_bound", st);
        if (col->key_bytes == 4)
            lower_bound_kernel<uint32_t><<<grid, 256, 0, st>>>(v, (const uint32_t*)vals, m, out);
        else
            lower_bound_kernel<uint64_t><<<grid, 256, 0, st>>>(v, (const uint64_t*)vals, m, out);
    }
    note_launch();
    return cuda_status(cudaGetLastError());
}

int quantile(const lc_column* col, const uint64_t* ks, uint64_t m, uint64_t q, int exact, void* out, cudaStream_t st) {
    if (m == 0) return LC_OK;
    const unsigned grid = (unsigned)std::min<uint64_t>((m + 255) / 256, (uint64_t)sm_count() * 16);
    {
        KTime kt(exact ? "quantile" : "quantile_approx", st);
        if (col->key_bytes == 4)
            quantile_kernel<uint32_t><<<grid, 256, 0, st>>>(col->view, ks, m, q, exact, (uint32_t*)out);
        else
            quantile_kernel<uint64_t><<<grid, 256, 0, st>>>(col->view, ks, m, q, exact, (uint64_t*)out);
    }
    note_launch();
    return cuda_status(cudaGetLastError());
}

int decode_approx(const lc_column* col, uint64_t begin, uint64_t count, void* out, cudaStream_t st) {
    if (count == 0) return LC_OK;
    const uint64_t t0 = host_tile_of(col, begin), nt = host_tile_of(col, begin + count - 1) - t0 + 1;
    const size_t smem = dec_smem(col->view.max_tile_segs);
    if (col->key_bytes == 4) {
        static DeviceOnce once;
        if (int rc = smem_attr_once(once, decode_approx_kernel<uint32_t>, kDecSmem)) return rc;
        const unsigned grid = (unsigned)std::min<uint64_t>(nt, dec_grid(decode_approx_kernel<uint32_t>, smem));
        KTime kt("decode_approx", st);
        decode_approx_kernel<uint32_t><<<grid, kDecThreads, smem, st>>>(col->view, t0, nt, begin, begin + count,
                                                                        (uint32_t*)out);
    } else {
        static DeviceOnce once;
        if (int rc = smem_attr_once(once, decode_approx_kernel<uint64_t>, kDecSmem)) return rc;
        const unsigned grid = (unsigned)std::min<uint64_t>(nt, dec_grid(decode_approx_kernel<uint64_t>, smem));
        KTime kt("decode_approx", st);
        decode_approx_kernel<uint64_t><<<grid, kDecThreads, smem, st>>>(col->view, t0, nt, begin, begin + count,
                                                                        (uint64_t*)out);
    }
    note_launch();
    return cuda_status(cudaGetLastError());
}

// Key and segment ranges of list l of a column (l < 0: the whole single column).
struct ListRange {
    uint64_t k0, k1, s0, s1;
};

static int list_range(const lc_column* col, int64_t l, cudaStream_t st, ListRange* r) {
    if (l < 0) {
        if (col->list_mode) return LC_ERR_INVALID_ARG;
        *r = ListRange{0, col->N, 0, col->L};
        return LC_OK;
    }
    if (!col->list_mode || (uint64_t)l >= col->NL) return LC_ERR_OUT_OF_RANGE;
    uint64_t kb[2], cb[2], sb[2];
    int rc = cuda_status(cudaMemcpyAsync(kb, col->blob + col->lay.lkb + 8 * l, 16, cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaMemcpyAsync(cb, col->blob + col->lay.lcb + 8 * l, 16, cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    if (!rc) rc = cuda_status(cudaMemcpyAsync(sb, col->blob + col->lay.csb + 8 * cb[0], 8, cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaMemcpyAsync(sb + 1, col->blob + col->lay.csb + 8 * cb[1], 8, cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    if (rc) return rc;
    *r = ListRange{kb[0], kb[1], sb[0], sb[1]};
    return LC_OK;
}

template <typename KT>
static int setop_t(bool is_and, const lc_column* a, const ListRange& ra, const lc_column* b, const ListRange& rb,
                   KT* out, uint64_t cap, uint64_t* count, cudaStream_t st) {
    const uint64_t nA = ra.k1 - ra.k0, nB = rb.k1 - rb.k0;
    // AND looks the shorter list up in the longer one
    const bool swap = is_and && nA > nB;
    const lc_column* cs = swap ? b : a;
    const lc_column* cl = swap ? a : b;
    const ListRange& rs = swap ? rb : ra;
    const ListRange& rl = swap ? ra : rb;
    const uint64_t n1 = rs.k1 - rs.k0, n2 = is_and ? 0 : rl.k1 - rl.k0;
    const uint64_t nflags = is_and ? n1 : (n1 + n2 + kMergeItems - 1) / kMergeItems;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t tmp_b = scan_tmp_bytes(nflags);
    const size_t o_s = 0, o_l = al(sizeof(KT) * n1), o_f = o_l + al(sizeof(KT) * n2), o_off = o_f + al(4 * nflags),
                 o_tmp = o_off + al(8 * (nflags + 1));
    uint8_t* p = nullptr;
    if (cudaMallocAsync((void**)&p, o_tmp + tmp_b + 16, st) != cudaSuccess) return LC_ERR_NOMEM;
    KT* S = (KT*)(p + o_s);
    KT* Lk = (KT*)(p + o_l);
    uint32_t* flag = (uint32_t*)(p + o_f);
    uint64_t* off = (uint64_t*)(p + o_off);
    int rc = decode_range(cs, rs.k0, n1, S, st);
    if (!rc && !is_and) rc = decode_range(cl, rl.k0, n2, Lk, st);
    const unsigned grid = (unsigned)std::min<uint64_t>((std::max<uint64_t>(nflags, 1) + 255) / 256, (uint64_t)sm_count() * 16);
    if (!rc && nflags) {
        KTime kt(is_and ? "and_probe" : "or_merge", st);
        if (is_and)
            and_flags_kernel<KT><<<grid, 256, 0, st>>>(cl->view, S, n1, rl.s0, rl.s1, rl.k0, rl.k1, flag);
        else
            or_merge_kernel<KT><<<grid, 256, 0, st>>>(S, n1, Lk, n2, 0, flag, nullptr, nullptr);
        note_launch();
        rc = cuda_status(cudaGetLastError());
    }
    if (!rc) rc = scan_exclusive(flag, off, nflags, ScanOp::Identity, p + o_tmp, tmp_b, st);
    uint64_t total = 0;
    if (!rc) rc = cuda_status(cudaMemcpyAsync(&total, off + nflags, 8, cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    if (!rc) {
        *count = total;
        if (total > cap || (total && !out)) rc = LC_ERR_INVALID_ARG;
    }
    if (!rc && total) {
        KTime kt(is_and ? "and_scatter" : "or_merge", st);
        if (is_and) scatter_flagged_kernel<KT><<<grid, 256, 0, st>>>(S, n1, flag, off, out);
        else or_merge_kernel<KT><<<grid, 256, 0, st>>>(S, n1, Lk, n2, 1, nullptr, off, out);
        note_launch();
        rc = cuda_status(cudaGetLastError());
    }
    cudaFreeAsync(p, st);
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    return rc;
}

int set_op(bool is_and, const lc_column* a, int64_t la, const lc_column* b, int64_t lb, void* out, uint64_t cap,
           uint64_t* count, cudaStream_t st) {
    if (a->key_bytes != b->key_bytes) return LC_ERR_INVALID_ARG;
    ListRange ra, rb;
    int rc = list_range(a, la, st, &ra);
    if (!rc) rc = list_range(b, lb, st, &rb);
    if (rc) return rc;
    if (a->key_bytes == 4) return setop_t<uint32_t>(is_and, a, ra, b, rb, (uint32_t*)out, cap, count, st);
    return setop_t<uint64_t>(is_and, a, ra, b, rb, (uint64_t*)out, cap, count, st);
}

// ------------------------------------------------------------------ multi-range decode without allocation
//
// lc_decode_ranges_noalloc serves callers that cannot call cudaMalloc or
// cudaMallocAsync: for example a serving loop that must keep the allocator (and
// the device synchronisation a cudaFree can imply) off its request path, or a
// host application that owns all device memory and gives libraries only
// buffers it allocated itself.  Its work lists live in one file-scope device
// array instead of a per-call allocation.  Every GPU that loads this library
// holds the array until the process exits.

namespace {

constexpr uint64_t kNoAllocMaxRanges = LC_NOALLOC_MAX_RANGES;
constexpr size_t kNoAllocFirstOff = 0;                                                // uint64 first[m]
constexpr size_t kNoAllocWorkOff = kNoAllocFirstOff + 8 * kNoAllocMaxRanges;          // uint64 work_off[m+1]
constexpr size_t kNoAllocTilesOff = (kNoAllocWorkOff + 8 * (kNoAllocMaxRanges + 1) + 255) & ~(size_t)255;
constexpr size_t kNoAllocScanOff = (kNoAllocTilesOff + 4 * kNoAllocMaxRanges + 255) & ~(size_t)255;
constexpr size_t kNoAllocScanBytes = 8 * ((kNoAllocMaxRanges + kScanTile - 1) / kScanTile + 1);  // scan partials
constexpr size_t kNoAllocScratchBytes = kNoAllocScanOff + kNoAllocScanBytes;

static_assert(kNoAllocScanBytes >= 8 * ((kNoAllocMaxRanges + kScanTile - 1) / kScanTile),
              "scan_exclusive needs one partial per scan tile");
__device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

uint8_t* g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
int noalloc_scratch(uint8_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return LC_ERR_INTERNAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e);
        g_noalloc_ptr[dev] = (uint8_t*)p;
    }
    *out = g_noalloc_ptr[dev];
    return LC_OK;
}

}  // namespace

int decode_ranges_noalloc(const lc_column* col, const uint64_t* begin, const uint64_t* count, const uint64_t* out_off,
                          uint64_t m, void* out, uint64_t out_cap, cudaStream_t st) {
    if (m > kNoAllocMaxRanges) return LC_ERR_INVALID_ARG;
    if (m == 0) return LC_OK;
    uint8_t* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    // Every word read below is written earlier in this call (first and ntiles
    // by range_tiles_kernel, the scan partials and work_off by the scan), so
    // nothing has to be cleared between calls.
    uint64_t* first = (uint64_t*)(scratch + kNoAllocFirstOff);
    uint64_t* work_off = (uint64_t*)(scratch + kNoAllocWorkOff);
    uint32_t* ntiles = (uint32_t*)(scratch + kNoAllocTilesOff);
    void* tmp = scratch + kNoAllocScanOff;
    range_tiles_kernel<<<(unsigned)std::min<uint64_t>((m + 255) / 256, 4096), 256, 0, st>>>(
        col->view, begin, count, out_off, out_cap, m, first, ntiles);
    note_launch();
    rc = cuda_status(cudaGetLastError());
    if (!rc) rc = scan_exclusive(ntiles, work_off, m, ScanOp::Identity, tmp, kNoAllocScanBytes, st);
    if (rc) return rc;
    const size_t smem = dec_smem(col->view.max_tile_segs);
    if (col->key_bytes == 4) {
        if ((rc = set_smem<uint32_t>())) return rc;
        decode_ranges_kernel<uint32_t><<<dec_grid(decode_ranges_kernel<uint32_t>, smem), kDecThreads, smem, st>>>(
            col->view, begin, count, out_off, m, first, work_off, (uint32_t*)out);
    } else {
        if ((rc = set_smem<uint64_t>())) return rc;
        decode_ranges_kernel<uint64_t><<<dec_grid(decode_ranges_kernel<uint64_t>, smem), kDecThreads, smem, st>>>(
            col->view, begin, count, out_off, m, first, work_off, (uint64_t*)out);
    }
    note_launch();
    return cuda_status(cudaGetLastError());
}


int serve_launch(const ColView* views_d, int key_bytes, const SrvReq* qreqs_d, uint32_t nqreq, uint64_t nq,
                 const uint64_t* qin_d, uint64_t* qout_d, const SrvReq* dreqs_d, uint32_t ndreq,
                 const uint64_t* work_off_d, uint64_t nwork, uint32_t max_tile_segs, uint32_t* status_d,
                 cudaStream_t st) {
    int rc;
    if (nq) {
        const unsigned grid = (unsigned)std::min<uint64_t>((nq + 255) / 256, (uint64_t)sm_count() * 8);
        if (key_bytes == 4)
            serve_query_kernel<uint32_t><<<grid, 256, 0, st>>>(views_d, qreqs_d, nqreq, nq, qin_d, qout_d, status_d);
        else
            serve_query_kernel<uint64_t><<<grid, 256, 0, st>>>(views_d, qreqs_d, nqreq, nq, qin_d, qout_d, status_d);
        note_launch();
        if ((rc = cuda_status(cudaGetLastError()))) return rc;
    }
    if (nwork) {
        const size_t smem = dec_smem(max_tile_segs);
        if (key_bytes == 4) {
            static DeviceOnce once;
            if ((rc = smem_attr_once(once, serve_decode_kernel<uint32_t>, kDecSmem))) return rc;
            const unsigned grid = (unsigned)std::min<uint64_t>(nwork, dec_grid(serve_decode_kernel<uint32_t>, smem));
            serve_decode_kernel<uint32_t><<<grid, kDecThreads, smem, st>>>(views_d, dreqs_d, ndreq, work_off_d,
                                                                          max_tile_segs);
        } else {
            static DeviceOnce once;
            if ((rc = smem_attr_once(once, serve_decode_kernel<uint64_t>, kDecSmem))) return rc;
            const unsigned grid = (unsigned)std::min<uint64_t>(nwork, dec_grid(serve_decode_kernel<uint64_t>, smem));
            serve_decode_kernel<uint64_t><<<grid, kDecThreads, smem, st>>>(views_d, dreqs_d, ndreq, work_off_d,
                                                                          max_tile_segs);
        }
        note_launch();
        if ((rc = cuda_status(cudaGetLastError()))) return rc;
    }
    return LC_OK;
}

uint64_t tile_of_key(const lc_column* col, uint64_t i) { return host_tile_of(col, i); }

int wait_selftest(uint32_t polls, cudaStream_t st) {
    uint32_t* d = nullptr;
    if (cudaMallocAsync((void**)&d, 4, st) != cudaSuccess) return LC_ERR_NOMEM;
    wait_selftest_kernel<<<1, 32, 0, st>>>(d, polls);
    note_launch();
    int rc = cuda_status(cudaGetLastError());
    uint32_t h = 0;
    if (!rc) rc = cuda_status(cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    cudaFreeAsync(d, st);
    if (rc) return rc;
    return (h & kStTimeout) ? LC_ERR_TIMEOUT : LC_OK;
}

}  // namespace lcx
