// lc_compress.cu -- the compression path on the GPU: eps-PLA fit (Def. 2,
// Eq. (1)), residual widths and packing (Sec. II-A), all in exact integer
// arithmetic so that the bytes equal those of the CPU definition.
//
// Pipeline for C chunks (each chunk is independent: segments never cross one):
//   spec_kernel   one CTA per window (4096 keys, 2048 for short lists), keys in shared memory;
//                 one thread per 64-key span runs the greedy from 96 keys
//                 before its span (a warm-up that almost always brings it onto
//                 the true chain) and records its anchors, entry and exit per
//                 32-key block.
//   chain_kernel  one warp per chunk follows the blocks in order: a ballot
//                 accepts every run of blocks whose walks join up, the warp
//                 walks the cone itself elsewhere (256 keys per step, 32-bit
//                 fractions where the keys allow); the true anchors as one bit
//                 per key, the segment count per chunk, and the slope of every
//                 segment longer than 96 keys (its walk ends with the cone).
//   scan          chunk_seg_begin.
//   fit_short_kernel  one CTA per window, one thread per 32-key
//                 block, split by keys: the cone, slope and width of every
//                 segment of at most 96 keys that starts in the block, with
//                 the keys of later blocks merged as partial cones through
//                 shared memory (keys in shared memory); longer segments queue
//                 their width pass.
//   long_width_kernel  one warp per 2048-key piece of a long segment.
//   bitoff_kernel one CTA per chunk: bit offsets (a scan of w (n-1)).
//   scan          chunk_word_begin.
//   pack_kernel   one CTA per chunk, 2048-key windows assembled in shared memory
//                 with shared atomics, then stored as whole 32-bit words.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lc_internal.h"
#include "lc_math.cuh"

namespace lcx {

// ceil(2^64 / d) for 2 <= d < 2^16 (entries 0 and 1 unused).
__device__ uint64_t g_magic[kMaxChunk];

namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;     // segment end not found within the walk limit
constexpr int kPackThreads = 256;
constexpr uint32_t kWin = 2048;             // keys per pack window
constexpr uint32_t kWalkAhead = 32 * 32;    // keys the warp walk prefetches into L2 ahead of its step

template <typename KT>
__device__ __forceinline__ uint64_t ldk(const KT* __restrict__ K, uint32_t i) {
    return (uint64_t)__ldg(K + i);
}

// Key i as a cone element relative to the anchor (x, kx): the real Q32
// slopes it admits are [2^32 (D - eps)/d, 2^32 (D + eps + 1)/d) (frac_step's
// reading).  A key whose lower bound reaches the int64 cap pins the lower
// bound above every upper one; a key past the chunk is the identity.
__device__ __forceinline__ Frac key_frac(uint64_t Ki, uint32_t i, uint32_t x, uint64_t kx, uint32_t n, int64_t eps) {
    Frac v;
    const uint32_t d = i - x;
    const uint64_t D = Ki - kx;
    if (i >= n) {
        v = frac_open();
    } else if (D < ((uint64_t)d << 31) + (uint64_t)eps) {
        v.X = (int64_t)D - eps;
        v.E = d;
        v.Y = D + (uint64_t)eps + 1;
        v.F = d;
    } else {
        v.X = (1ll << 47) - 1;
        v.E = 1;
        v.Y = 1ull << 31;
        v.F = 1;
    }
    return v;
}

// Intersection of two cones: the larger lower fraction, the smaller upper.
__device__ __forceinline__ void frac_meet(Frac& v, const Frac& o) {
    if (frac_gt(o.X, o.E, v.X, v.E)) { v.X = o.X; v.E = o.E; }
    if (o.Y * (uint64_t)v.F < v.Y * (uint64_t)o.F) { v.Y = o.Y; v.F = o.F; }
}

__device__ __forceinline__ Frac shfl_frac(const Frac& v, int src) {
    Frac f;
    f.X = __shfl_sync(0xFFFFFFFFu, v.X, src);
    f.E = __shfl_sync(0xFFFFFFFFu, v.E, src);
    f.Y = __shfl_sync(0xFFFFFFFFu, v.Y, src);
    f.F = __shfl_sync(0xFFFFFFFFu, v.F, src);
    return f;
}

// The cone of frac_step with 32-bit numerators, for walks whose key range
// (plus eps + 1) stays below 2^31: then every D - eps and D + eps + 1 fits in
// an int32 and every cross product in 48 bits, and the int64 cap on the
// slope (2^31 per key) can never be reached.  Same decisions as frac_step.
struct Frac32 {
    int32_t X;
    uint32_t E;
    uint32_t Y;
    uint32_t F;
};
__device__ __forceinline__ Frac32 frac32_open() { return Frac32{INT32_MIN, 1u, 0x7FFFFFFFu, 1u}; }

constexpr uint32_t kWalkLane = 8;                 // keys per lane in one step of the warp walk
constexpr uint32_t kWalkStep = 32 * kWalkLane;    // 256 keys per step

// The walk's cone arithmetic in two widths with the same decisions: 64-bit
// (Frac) in general, 32-bit numerators (Frac32) for a step whose keys all lie
// less than 2^31 - eps - 1 above the anchor, where every numerator fits an
// int32 and every cross product 48 bits (and no key reaches the int64 cap).
// The open cone is -2^31/1 .. 2^31/1 in both.
struct WalkWide {
    using F = Frac;
    static __device__ __forceinline__ F open() { return frac_open(); }
    static __device__ __forceinline__ F key(uint64_t Ki, uint32_t i, uint32_t x, uint64_t kx, uint32_t n, int64_t eps) {
        return key_frac(Ki, i, x, kx, n, eps);
    }
    static __device__ __forceinline__ void meet(F& v, const F& o) { frac_meet(v, o); }
    static __device__ __forceinline__ bool ok(const F& c) { return frac_ok(c); }
    static __device__ __forceinline__ F shfl(const F& v, int src) { return shfl_frac(v, src); }
    static __device__ __forceinline__ F shfl_up(const F& v, int off) {
        F o;
        o.X = __shfl_up_sync(0xFFFFFFFFu, v.X, off);
        o.E = __shfl_up_sync(0xFFFFFFFFu, v.E, off);
        o.Y = __shfl_up_sync(0xFFFFFFFFu, v.Y, off);
        o.F = __shfl_up_sync(0xFFFFFFFFu, v.F, off);
        return o;
    }
    static __device__ __forceinline__ F from(const Frac& f) { return f; }
    static __device__ __forceinline__ Frac wide(const F& f) { return f; }
};
struct WalkNarrow {
    using F = Frac32;
    static __device__ __forceinline__ F open() { return Frac32{INT32_MIN, 1u, 0x80000000u, 1u}; }
    static __device__ __forceinline__ F key(uint64_t Ki, uint32_t i, uint32_t x, uint64_t kx, uint32_t n, int64_t eps) {
        if (i >= n) return open();
        const uint32_t D = (uint32_t)(Ki - kx), d = i - x;
        return Frac32{(int32_t)D - (int32_t)eps, d, D + (uint32_t)eps + 1u, d};
    }
    static __device__ __forceinline__ void meet(F& v, const F& o) {
        if ((int64_t)o.X * v.E > (int64_t)v.X * o.E) { v.X = o.X; v.E = o.E; }
        if ((uint64_t)o.Y * v.F < (uint64_t)v.Y * o.F) { v.Y = o.Y; v.F = o.F; }
    }
    static __device__ __forceinline__ bool ok(const F& c) {
        return c.X < 0 || (uint64_t)(uint32_t)c.X * c.F < (uint64_t)c.Y * c.E;
    }
    static __device__ __forceinline__ F shfl(const F& v, int src) {
        return Frac32{__shfl_sync(0xFFFFFFFFu, v.X, src), __shfl_sync(0xFFFFFFFFu, v.E, src),
                      __shfl_sync(0xFFFFFFFFu, v.Y, src), __shfl_sync(0xFFFFFFFFu, v.F, src)};
    }
    static __device__ __forceinline__ F shfl_up(const F& v, int off) {
        return Frac32{__shfl_up_sync(0xFFFFFFFFu, v.X, off), __shfl_up_sync(0xFFFFFFFFu, v.E, off),
                      __shfl_up_sync(0xFFFFFFFFu, v.Y, off), __shfl_up_sync(0xFFFFFFFFu, v.F, off)};
    }
    static __device__ __forceinline__ F from(const Frac& f) { return Frac32{(int32_t)f.X, f.E, (uint32_t)f.Y, f.F}; }
    static __device__ __forceinline__ Frac wide(const F& f) {
        return Frac{(int64_t)f.X, f.E, (uint64_t)f.Y, f.F};
    }
};

// One step of the warp walk over keys p .. p + 255 (cur: lane l's keys
// p + 8l .. p + 8l + 7): lane l intersects the slope intervals of its keys,
// an inclusive scan over the lanes gives the cone after every lane's keys,
// and the first lane whose cone is empty holds the next anchor, which that
// lane finds key by key from the cone before it.  Returns true with the
// anchor in *end and the segment's cone in *fin when the segment ends in
// this step; else carries the cone on and returns false.
template <typename W>
__device__ __forceinline__ bool walk_step(const uint64_t (&cur)[kWalkLane], uint32_t p, uint32_t x, uint64_t kx,
                                          uint32_t n, int64_t eps, uint32_t lane, Frac& carried, uint32_t* end,
                                          Frac* fin) {
    using F = typename W::F;
    const F cone = W::from(carried);
    const uint32_t i0 = p + kWalkLane * lane;
    F v = W::open();
#pragma unroll
    for (uint32_t u = 0; u < kWalkLane; ++u) W::meet(v, W::key(cur[u], i0 + u, x, kx, n, eps));
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const F o = W::shfl_up(v, off);
        if (lane >= (uint32_t)off) W::meet(v, o);
    }
    W::meet(v, cone);
    const uint32_t badm = __ballot_sync(0xFFFFFFFFu, !W::ok(v));
    if (badm) {
        const int bl = __ffs(badm) - 1;
        const F before = W::shfl(v, bl > 0 ? bl - 1 : 0);
        F c = bl > 0 ? before : cone;
        uint32_t brk = 0;
        if (lane == (uint32_t)bl) {
            brk = kWalkLane;
#pragma unroll
            for (uint32_t u = 0; u < kWalkLane; ++u) {
                if (brk != kWalkLane) continue;
                F t = c;
                W::meet(t, W::key(cur[u], i0 + u, x, kx, n, eps));
                if (!W::ok(t)) brk = u;
                else c = t;
            }
        }
        brk = __shfl_sync(0xFFFFFFFFu, brk, bl);
        *fin = W::wide(W::shfl(c, bl));
        *end = min(p + kWalkLane * (uint32_t)bl + brk, n);
        return true;
    }
    carried = W::wide(W::shfl(v, 31));
    return false;
}

// The greedy cone (Def. 2, shrinking-cone reading) with a whole warp, 256
// keys per step (walk_step); the keys of the next step are loaded while this
// one computes, and a step runs in 32-bit fractions when its keys allow.
// Called with all 32 lanes active and warp-uniform arguments.  *fin
// receives the cone of the segment's keys (every lane).
template <typename KT>
__device__ __forceinline__ uint32_t warp_walk(const KT* __restrict__ K, uint32_t x, uint32_t n, int64_t eps, uint32_t lane,
                              Frac* fin) {
    const uint64_t kx = ldk(K, x);
    Frac cone = frac_open();
    uint32_t p = x + 1;
    uint64_t cur[kWalkLane], nxt[kWalkLane];
#pragma unroll
    for (uint32_t u = 0; u < kWalkLane; ++u) {
        const uint32_t i = p + kWalkLane * lane + u;
        nxt[u] = i < n ? ldk(K, i) : 0;
    }
    while (p < n) {
#pragma unroll
        for (uint32_t u = 0; u < kWalkLane; ++u) cur[u] = nxt[u];
        const uint32_t pn = p + kWalkStep;
        if (pn < n) {
#pragma unroll
            for (uint32_t u = 0; u < kWalkLane; ++u) {
                const uint32_t i = pn + kWalkLane * lane + u;
                nxt[u] = i < n ? ldk(K, i) : 0;
            }
            if (pn + kWalkAhead < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(K + pn + kWalkAhead + 8 * lane));
        }
        // the lane's largest key offset (keys are sorted: its last key in the chunk)
        const uint32_t i0 = p + kWalkLane * lane;
        uint64_t dmax = 0;
#pragma unroll
        for (uint32_t u = 0; u < kWalkLane; ++u)
            if (i0 + u < n) dmax = cur[u] - kx;
        const bool narrow = __all_sync(0xFFFFFFFFu, dmax + (uint64_t)eps + 1 < (1ull << 31));
        uint32_t end = 0;
        if (narrow ? walk_step<WalkNarrow>(cur, p, x, kx, n, eps, lane, cone, &end, fin)
                   : walk_step<WalkWide>(cur, p, x, kx, n, eps, lane, cone, &end, fin))
            return end;
        p = pn;
    }
    *fin = cone;
    return n;
}

// ------------------------------------------------------------------ fit: speculation with a warm-up walk

constexpr uint32_t kFB = 32;                    // keys per fit block: one 32-bit word of anchor bits
constexpr uint32_t kWarm = 96;                  // keys a speculative walk runs before its span
constexpr int kChainThreads = 128;              // four chunks per CTA, one warp each
constexpr uint32_t kShortMax = 96;              // segments of at most this many keys: one thread fits each
static_assert(kShortMax == 96, "the speculative walks and fit_short_kernel's anchor search assume 96");

// Keys per window (one CTA of spec_kernel, fit_short_kernel and reach_kernel).
// A window never spans two chunks, so chunks shorter than a window leave its
// threads idle: columns of short lists take 2048-key windows (at the default
// span, 32 speculating threads), long chunks 4096 (more CTAs per chunk than
// 8192 without more warm-up per key; both measured faster than 8192).
constexpr uint32_t kWinWide = 4096, kWinNarrow = 2048;
template <uint32_t WK>
struct Win {
    static constexpr uint32_t kSpecKeys = kWarm + WK + 96;  // a walk ends at most 96 keys past its span
    static constexpr uint32_t kSpecSlots = kSpecKeys + kSpecKeys / 32 + 1;  // the densest padding (one per 32 keys)
    static constexpr int kShortThreads = WK / kFB;         // one thread per 32-key block in fit_short_kernel
    static constexpr uint32_t kLongPerWin = WK / (kShortMax + 1) + 1;  // segments > 96 keys starting in a window
    static constexpr uint32_t kShortSlots = (WK + kShortMax) + (WK + kShortMax) / 32 + 1;
    static_assert(kShortThreads % 32 == 0, "whole warps");
};
constexpr uint32_t kPiece = 2048;               // keys per work item of a long segment's width pass

// A segment longer than kShortMax keys, as its walk in the chain found it.
struct LongInfo {
    int64_t M;     // slope
    uint32_t end;  // next anchor (chunk-relative) or the chunk's length
    uint32_t pad;
};
// The width pass of one long segment: keys key0 + [1, n), running max of the
// zigzag residuals in zmax.
struct LongItem {
    uint64_t key0;
    int64_t M;
    uint32_t n;
    uint32_t zmax;
    uint64_t pad;
};
// A long segment met by a window of fit_short_kernel: segment j, anchored at
// chunk position a, len keys, slope M; its pieces start at poff in the window.
struct WinLong {
    uint64_t j;
    int64_t M;
    uint32_t a, len, poff, pad;
};
// Keys key0 + [t0, t1) of long segment `item`.
struct Piece {
    uint32_t item;
    uint32_t t0, t1;
    uint32_t pad;
};

// A window's keys staged in shared memory: local key q sits in slot q + q/32,
// so that lanes walking 32 consecutive 32-key blocks read distinct banks.
template <typename KT>
struct Staged {
    const KT* s;
    uint32_t base;
    __device__ __forceinline__ uint64_t operator()(uint32_t i) const {
        const uint32_t q = i - base;
        return (uint64_t)s[q + (q >> 5)];
    }
};


// What one speculative walk leaves for its kB 32-key blocks: its anchors in
// each block (m), and e[k] = its first anchor at or after the start of block k
// (e[0]: the span's start = entry of block 0; e[kB]: the span's end = exit of
// the last block); kNone where the walk stopped before finding it.
template <int kB>
struct SpecOut {
    uint32_t m[kB];
    uint32_t e[kB + 1];
};

template <int kB>
__device__ __forceinline__ void spec_record(SpecOut<kB>& o, uint32_t i, uint32_t s0) {
    const uint32_t r = i - s0;
#pragma unroll
    for (int k = 0; k < kB; ++k)
        if (r >= 32u * k && r < 32u * (k + 1)) o.m[k] |= 1u << (r - 32u * k);
#pragma unroll
    for (int k = 0; k <= kB; ++k)
        if (o.e[k] == kNone && r >= 32u * k) o.e[k] = i;
}

// One thread's speculative walk: the greedy from `p` (taken as an anchor)
// until its first anchor at or after s0 + 32 kB (the span's end) or the
// chunk's end n.  A segment that would grow past kShortMax keys stops it (its
// end is left to the chain, which walks long segments itself), so every
// segment the walk closes has at most kShortMax keys.  The narrow walk reads
// 32-bit key offsets from shared memory (exact differences: the walk's key
// range is below 2^31); the wide one reads 64-bit keys from global memory.
template <bool kNarrow, int kB, typename ST>
__device__ __forceinline__ SpecOut<kB> spec_walk(const ST& st, uint32_t p, uint32_t n, uint32_t s0, int64_t eps) {
    constexpr uint32_t kSpanB = 32u * kB;
    SpecOut<kB> o;
#pragma unroll
    for (int k = 0; k < kB; ++k) o.m[k] = 0u;
#pragma unroll
    for (int k = 0; k <= kB; ++k) o.e[k] = kNone;
    const uint32_t lim = min(n, s0 + kSpanB + kShortMax);
    uint32_t x = p;
    if (p >= s0) spec_record<kB>(o, p, s0);
    uint32_t i = p + 1;
    if (kNarrow) {
        // branch-free steps: every lane runs the same instructions whether its
        // key moves the cone, leaves it alone or starts a new segment
        uint32_t kx = (uint32_t)st(p);
        int32_t X = INT32_MIN;
        uint32_t E = 1u, Y = 0x7FFFFFFFu, F = 1u;
        const int32_t e32 = (int32_t)eps;
        for (; i < lim && i - x <= kShortMax; ++i) {
            const uint32_t Ki = (uint32_t)st(i);
            const uint32_t D = Ki - kx, d = i - x;
            const int32_t xl = (int32_t)D - e32;
            const uint32_t yh = D + (uint32_t)e32 + 1u;
            const bool lm = (int64_t)xl * E > (int64_t)X * d;
            const bool hm = (uint64_t)yh * F < (uint64_t)Y * d;
            const int32_t nX = lm ? xl : X;
            const uint32_t nE = lm ? d : E, nY = hm ? yh : Y, nF = hm ? d : F;
            const bool ok = nX < 0 || (uint64_t)(uint32_t)nX * nF < (uint64_t)nY * nE;
            X = ok ? nX : INT32_MIN;
            E = ok ? nE : 1u;
            Y = ok ? nY : 0x7FFFFFFFu;
            F = ok ? nF : 1u;
            if (!ok) {
                x = i;
                kx = Ki;
                if (i >= s0) {
                    spec_record<kB>(o, i, s0);
                    if (i >= s0 + kSpanB) break;
                }
            }
        }
    } else {
        uint64_t kx = st(p);
        Frac c = frac_open();
        for (; i < lim && i - x <= kShortMax; ++i) {
            const uint64_t Ki = st(i);
            if (frac_step(Ki - kx, i - x, eps, c)) continue;
            x = i;
            kx = Ki;
            c = frac_open();
            if (i >= s0) {
                spec_record<kB>(o, i, s0);
                if (i >= s0 + kSpanB) break;
            }
        }
    }
    // the walk ran into the chunk's end inside a segment of at most kShortMax keys: n is its next anchor
    if (i >= n && i - x <= kShortMax) {
#pragma unroll
        for (int k = 0; k <= kB; ++k)
            if (o.e[k] == kNone) o.e[k] = n;
    }
    return o;
}

// A window's keys staged in shared memory with one pad slot per 2^kShift keys,
// for lanes 2^kShift keys apart (distinct banks).
template <typename KT, int kShift>
struct StagedS {
    const KT* s;
    uint32_t base;
    __device__ __forceinline__ uint64_t operator()(uint32_t i) const {
        const uint32_t q = i - base;
        return (uint64_t)s[q + (q >> kShift)];
    }
};

// Key i of a chunk from global memory (the wide speculative walk).
template <typename KT>
struct GlobalKeys {
    const KT* K;
    __device__ __forceinline__ uint64_t operator()(uint32_t i) const { return (uint64_t)__ldg(K + i); }
};

// One CTA per window of WK keys of one chunk; keys [w0 - kWarm, w1 + 96)
// staged in shared memory as 32-bit offsets from the first staged key.
// Thread t owns the span of blocks kB t .. kB t + kB - 1 (32 kB keys) and runs
// the greedy from kWarm keys before the span (from the chunk start if that is
// closer) to its first anchor past the span.  Greedy walks from different
// starts meet after a few segments, so by the span the walk is almost always
// on the true chain; the chain kernel checks that (a block is exact iff the
// walk enters it where the previous block's walk leaves it) and walks itself
// where it does not hold.  Per block: the walk's anchors in the block (spec),
// its first anchor at or after the block's start (entry) and after its end
// (exit); kNone if the walk stopped inside a segment of more than kShortMax
// keys before reaching it, the chunk's length if the chunk ends first.  Also
// checks sortedness.  kB (1, 2 or 4 blocks per thread: WK / 32, WK / 64 or
// WK / 128 threads per window of WK keys) trades parallelism against the
// warm-up walked per key.
template <typename KT, int kB, uint32_t WK>
__global__ void __launch_bounds__(WK / (32 * kB))
spec_kernel(const KT* __restrict__ keys, const ChunkDesc* __restrict__ chunks, const WinDesc* __restrict__ wins,
            uint32_t* __restrict__ spec_g, uint32_t* __restrict__ entry_g, uint32_t* __restrict__ exit_g,
            uint32_t* __restrict__ status) {
    constexpr uint32_t kSpanB = 32u * kB;
    constexpr int kThreads = WK / kSpanB;
    static_assert(kThreads % 32 == 0, "whole warps");
    constexpr int kShift = kB == 1 ? 5 : (kB == 2 ? 6 : 7);
    extern __shared__ __align__(16) uint8_t smem[];
    const WinDesc wd = wins[blockIdx.x];
    const ChunkDesc cd = chunks[wd.chunk];
    const KT* __restrict__ K = keys + cd.key_begin;
    const uint32_t n = cd.n, w0 = wd.off, w1 = min(n, w0 + WK);
    const int64_t eps = cd.eps;
    const uint32_t tid = threadIdx.x;
    const uint32_t base = w0 >= kWarm ? w0 - kWarm : 0;
    const uint32_t top = min(n, w1 + 96);
    // stage the low 32 bits of K[i] - K[base]: a difference of two staged
    // values is exact whenever the true difference is below 2^32
    uint32_t* s = (uint32_t*)smem;
    const uint64_t kbase = (uint64_t)__ldg(K + base);
#pragma unroll 4
    for (uint32_t q = tid; q < top - base; q += kThreads)
        s[q + (q >> kShift)] = (uint32_t)((uint64_t)__ldg(K + base + q) - kbase);
    // sortedness: key i against key i - 1 for i in [max(w0, 1), w1)
    bool unsorted = false;
#pragma unroll 4
    for (uint32_t i = max(w0, 1u) + tid; i < w1; i += kThreads) unsorted |= __ldg(K + i - 1) > __ldg(K + i);
    if (w0 == 0 && cd.check_prev && tid == 0) unsorted |= __ldg(K - 1) > __ldg(K);
    if (unsorted) atomicOr(status, kStUnsorted);
    __syncthreads();
    const StagedS<uint32_t, kShift> st{s, base};

    const uint32_t s0 = w0 + tid * kSpanB;  // this thread's span [s0, s0 + 32 kB) (may start past w1)
    const bool active = s0 < w1;
    const uint32_t p = s0 >= base + kWarm ? s0 - kWarm : base;
    const uint32_t lim = active ? min(n, s0 + kSpanB + kShortMax) : p + 1;
    // the walk may use 32-bit numerators when its whole key range allows it (warp-uniform choice)
    const uint64_t span_keys = active ? (uint64_t)__ldg(K + lim - 1) - (uint64_t)__ldg(K + p) : 0;
    const bool narrow = __all_sync(0xFFFFFFFFu, span_keys + (uint64_t)eps + 1 < (1ull << 31));
    if (!active) return;
    const SpecOut<kB> o = narrow ? spec_walk<true, kB>(st, p, n, s0, eps)
                                 : spec_walk<false, kB>(GlobalKeys<KT>{K}, p, n, s0, eps);
    const uint64_t g = cd.bitword_begin + s0 / kFB;
#pragma unroll
    for (int k = 0; k < kB; ++k) {
        const uint32_t b0 = s0 + kFB * k;
        if (b0 >= w1) break;
        const uint32_t e = min(b0 + kFB, n);
        spec_g[g + k] = o.m[k] & (e - b0 < 32 ? (1u << (e - b0)) - 1u : 0xFFFFFFFFu);
        entry_g[g + k] = o.e[k];
        exit_g[g + k] = o.e[k + 1];
    }
}

// ------------------------------------------------------------------ fit: the true chain

// One warp per chunk follows the true anchors block by block.  At an exact
// anchor x of block k that the speculative walk of block k also passes
// through, the walk is exact from x on; the blocks after it stay exact as long
// as each one's walk enters where the previous one's leaves (a ballot over 32
// blocks takes the whole run at once).  Elsewhere the warp walks one segment
// itself (32 keys per step, or 256 while the cone does not move) and looks
// again.  Output: the chunk's anchor bitmap and segment count.  Every segment
// longer than kShortMax keys is found by such a walk (a speculative walk stops
// inside any segment longer than that), and the walk ends with the segment's
// cone: its slope and end are recorded at the anchor's block (at most one such
// segment starts in a block).
template <typename KT>
__global__ void __launch_bounds__(kChainThreads, 6)
chain_kernel(const KT* __restrict__ keys, const ChunkDesc* __restrict__ chunks, uint64_t C,
             const uint32_t* __restrict__ spec_g, const uint32_t* __restrict__ entry_g,
             const uint32_t* __restrict__ exit_g, uint32_t* __restrict__ tbits, uint32_t* __restrict__ counts,
             LongInfo* __restrict__ longinfo) {
    const uint64_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    if (c >= C) return;  // whole warps leave together
    const uint32_t lane = threadIdx.x & 31u;
    const ChunkDesc cd = chunks[c];
    const KT* __restrict__ K = keys + cd.key_begin;
    const uint32_t n = cd.n, nblk = (n + kFB - 1) / kFB;
    const int64_t eps = cd.eps;
    const uint64_t gb = cd.bitword_begin;
    uint32_t* __restrict__ T = tbits + gb;
    const uint64_t* __restrict__ magic = g_magic;
    // walk the segment anchored at a; record it when it is long
    auto walk = [&](uint32_t a) {
        Frac f;
        const uint32_t e = warp_walk(K, a, n, eps, lane, &f);
        if (e - a > kShortMax && lane == 0) longinfo[gb + (a >> 5)] = LongInfo{frac_slope(f, magic), e, 0u};
        return e;
    };
    uint32_t x = 0, knext = 0, total = 0, pm = 0;  // pm: anchors of block knext found so far
    while (x < n) {
        const uint32_t k = x / kFB, b = k * kFB;
        if (k != knext) pm = 0;
        for (uint32_t q = knext + lane; q < k; q += 32) T[q] = 0;
        knext = k;
        // the walks of blocks k .. k+31 (one load round per step)
        const uint32_t kb = k + lane;
        const bool valid = kb < nblk;
        uint32_t m = 0, ex = kNone, ent = kNone;
        if (valid) {
            m = __ldg(spec_g + gb + kb);
            ex = __ldg(exit_g + gb + kb);
            ent = __ldg(entry_g + gb + kb);
        }
        const uint32_t m0 = __shfl_sync(0xFFFFFFFFu, m, 0);
        if ((m0 >> (x - b)) & 1u) {
            // x is on block k's walk: exact from x on; extend over consistent blocks
            if (lane == 0) m = pm | (m & (0xFFFFFFFFu << (x - b)));
            const uint32_t exp = __shfl_up_sync(0xFFFFFFFFu, ex, 1);
            const bool cons = valid && (lane == 0 || (ent == exp && exp != kNone));
            const uint32_t okm = __ballot_sync(0xFFFFFFFFu, cons);
            const uint32_t r = ~okm ? (uint32_t)__ffs(~okm) - 1u : 32u;  // lanes 0..r-1 follow one another (r >= 1)
            if (lane < r) T[kb] = m;
            total += __reduce_add_sync(0xFFFFFFFFu, lane < r ? (uint32_t)__popc(m) : 0u);
            uint32_t xl = __shfl_sync(0xFFFFFFFFu, ex, r - 1);
            if (xl == kNone) {
                // the last walk stopped inside a segment: walk it from its anchor
                const uint32_t nz = __ballot_sync(0xFFFFFFFFu, lane < r && m != 0u);  // lane 0 holds x: nz != 0
                const uint32_t h = 31u - (uint32_t)__clz(nz);
                const uint32_t mh = __shfl_sync(0xFFFFFFFFu, m, h);
                xl = walk((k + h) * kFB + 31u - (uint32_t)__clz(mh));
            }
            knext = k + r;
            pm = 0;
            x = xl;
        } else {
            // walk one segment from x and look again
            pm |= 1u << (x - b);
            const uint32_t xn = walk(x);
            if (xn >= b + kFB || xn >= n) {
                if (lane == 0) T[k] = pm;
                total += __popc(pm);
                knext = k + 1;
                pm = 0;
            }
            x = xn;
        }
    }
    for (uint32_t q = knext + lane; q < nblk; q += 32) T[q] = 0;
    if (lane == 0) counts[c] = total;
}

// ------------------------------------------------------------------ the jump fit (fewest segments)
//
// Sec. II-A fits with the fewest segments.  Every feasible anchored segment is
// a prefix of the greedy one from its anchor, so the fewest segments follow
// from each position's greedy reach r(p) by the jump-game choice: from anchor
// a, end the segment at the position in (a, r(a)] whose own reach is
// farthest.  Reaches are taken up to kShortMax keys (r(p) "long" beyond; a
// long reach counts as farthest, ties go to the first position), a long
// segment is walked as by the greedy, and a chunk keeps the jump segmentation
// only if it has fewer segments than the greedy's.

// reach_kernel: one CTA per window of WK keys, keys [w0, w1 + 96] staged as
// 32-bit offsets; r_off[p] = r(p) - p in 1..96, or 0 when the greedy segment
// from p is longer than 96 keys.  One thread per position.
template <typename KT, uint32_t WK>
__global__ void __launch_bounds__(Win<WK>::kShortThreads)
reach_kernel(const KT* __restrict__ keys, const ChunkDesc* __restrict__ chunks, const WinDesc* __restrict__ wins,
             uint8_t* __restrict__ roff) {
    constexpr int kThr = Win<WK>::kShortThreads;
    extern __shared__ __align__(16) uint8_t smem[];
    const WinDesc wd = wins[blockIdx.x];
    const ChunkDesc cd = chunks[wd.chunk];
    const KT* __restrict__ K = keys + cd.key_begin;
    const uint32_t n = cd.n, w0 = wd.off, w1 = min(n, w0 + WK);
    const int64_t eps = cd.eps;
    const uint32_t top = min(n, w1 + kShortMax + 1);
    uint32_t* s = (uint32_t*)smem;
    const uint64_t kbase = (uint64_t)__ldg(K + w0);
#pragma unroll 4
    for (uint32_t q = threadIdx.x; q < top - w0; q += kThr)
        s[q + (q >> 5)] = (uint32_t)((uint64_t)__ldg(K + w0 + q) - kbase);
    __syncthreads();
    const Staged<uint32_t> st{s, w0};
    const uint32_t iters = (w1 - w0 + kThr - 1) / kThr;  // the same for every thread
    for (uint32_t it = 0; it < iters; ++it) {
        const uint32_t p = w0 + threadIdx.x + it * kThr;
        const bool active = p < w1;
        const uint32_t lim = active ? min(n, p + kShortMax + 1) : p + 1;
        const uint64_t span = active ? (uint64_t)__ldg(K + lim - 1) - (uint64_t)__ldg(K + p) : 0;
        const bool narrow = __all_sync(0xFFFFFFFFu, span + (uint64_t)eps + 1 < (1ull << 31));
        if (!active) continue;
        uint32_t i = p + 1;
        if (narrow) {
            const uint32_t kx = (uint32_t)st(p);
            int32_t X = INT32_MIN;
            uint32_t E = 1u, Y = 0x7FFFFFFFu, F = 1u;
            const int32_t e32 = (int32_t)eps;
            for (; i < lim; ++i) {
                const uint32_t D = (uint32_t)st(i) - kx, d = i - p;
                const int32_t xl = (int32_t)D - e32;
                const uint32_t yh = D + (uint32_t)e32 + 1u;
                if ((int64_t)xl * E > (int64_t)X * d) { X = xl; E = d; }
                if ((uint64_t)yh * F < (uint64_t)Y * d) { Y = yh; F = d; }
                if (X >= 0 && (uint64_t)(uint32_t)X * F >= (uint64_t)Y * E) break;
            }
        } else {
            const uint64_t kx = (uint64_t)__ldg(K + p);
            Frac c = frac_open();
            for (; i < lim; ++i)
                if (!frac_step((uint64_t)__ldg(K + i) - kx, i - p, eps, c)) break;
        }
        // i: the first key that empties the cone, or lim (the chunk's end, or 97 keys on)
        roff[cd.key_begin + p] = (uint8_t)(i - p <= kShortMax ? i - p : 0u);
    }
}

// jump_kernel: one warp per chunk; the reaches of 256 positions at a time sit
// in the lanes (8 bytes each).  Writes the jump segmentation's anchor bits and
// long-segment records to scratch, then replaces the greedy's for the chunk
// when it has fewer segments.
template <typename KT>
__global__ void __launch_bounds__(kChainThreads, 6)
jump_kernel(const KT* __restrict__ keys, const ChunkDesc* __restrict__ chunks, uint64_t C,
            const uint8_t* __restrict__ roff, uint32_t* __restrict__ tbits, uint32_t* __restrict__ counts,
            LongInfo* __restrict__ longinfo, uint32_t* __restrict__ jbits, LongInfo* __restrict__ jlong) {
    const uint64_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    if (c >= C) return;
    const uint32_t lane = threadIdx.x & 31u;
    const ChunkDesc cd = chunks[c];
    const KT* __restrict__ K = keys + cd.key_begin;
    const uint8_t* __restrict__ R = roff + cd.key_begin;
    const uint32_t n = cd.n, nblk = (n + kFB - 1) / kFB;
    const int64_t eps = cd.eps;
    const uint64_t gb = cd.bitword_begin;
    uint32_t* __restrict__ J = jbits + gb;
    const uint64_t* __restrict__ magic = g_magic;
    for (uint32_t q = lane; q < nblk; q += 32) J[q] = 0;
    __syncwarp();
    auto load_win = [&](uint32_t base) {
        uint64_t v = 0;
#pragma unroll
        for (uint32_t u = 0; u < 8; ++u) {
            const uint32_t q = base + 8 * lane + u;
            v |= (uint64_t)(q < n ? R[q] : 0) << (8 * u);
        }
        return v;
    };
    uint32_t base = 0;
    uint64_t win = load_win(0);
    uint32_t a = 0, cnt = 0;
    while (a < n) {
        ++cnt;
        if (lane == 0) J[a >> 5] |= 1u << (a & 31u);
        if (a + kShortMax >= base + 256) {  // the window must hold positions a .. a + 96
            base = a;
            win = load_win(base);
        }
        const uint32_t oa = a - base;
        const uint32_t ra = (uint32_t)(__shfl_sync(0xFFFFFFFFu, win, oa >> 3) >> (8 * (oa & 7u))) & 0xFFu;
        uint32_t nx;
        if (ra == 0) {  // the greedy segment from a is long: walk it
            Frac f;
            nx = warp_walk(K, a, n, eps, lane, &f);
            if (lane == 0) jlong[gb + (a >> 5)] = LongInfo{frac_slope(f, magic), nx, 0u};
        } else if (a + ra >= n) {
            nx = n;
        } else {
            // the candidate in (a, a + ra] that reaches farthest (long: farthest; ties: the first)
            const uint32_t hi = a + ra;
            uint32_t bv = 0, bq = 0xFFFFFFFFu;
#pragma unroll
            for (uint32_t u = 0; u < 8; ++u) {
                const uint32_t q = base + 8 * lane + u;
                if (q > a && q <= hi) {
                    const uint32_t r = (uint32_t)(win >> (8 * u)) & 0xFFu;
                    const uint32_t v = r ? q + r : 0xFFFFFFFFu;
                    if (v > bv) {
                        bv = v;
                        bq = q;
                    }
                }
            }
            const uint32_t mv = __reduce_max_sync(0xFFFFFFFFu, bv);
            nx = __reduce_min_sync(0xFFFFFFFFu, bv == mv ? bq : 0xFFFFFFFFu);
        }
        a = nx;
    }
    __syncwarp();
    const bool better = cnt < __ldg(counts + c);
    if (better) {
        uint32_t* __restrict__ T = tbits + gb;
        for (uint32_t q = lane; q < nblk; q += 32) {
            T[q] = J[q];
            longinfo[gb + q] = jlong[gb + q];  // read only at long anchors, which the jump recorded
        }
        if (lane == 0) counts[c] = cnt;
    }
}

// ------------------------------------------------------------------ block scans

template <typename T, typename Op>
__device__ __forceinline__ T warp_incl_scan(T v, Op op, uint32_t lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        T o = __shfl_up_sync(0xFFFFFFFFu, v, off);
        if (lane >= (uint32_t)off) v = op(v, o);
    }
    return v;
}

// Exclusive block scan (blockDim.x a multiple of 32, <= 1024); returns the
// exclusive prefix of v and writes the block total to *total.
template <typename T, typename Op>
__device__ T block_excl_scan(T v, Op op, T ident, T* s_warp, T* total) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_incl_scan(v, op, lane);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? s_warp[lane] : ident;
        T wi = warp_incl_scan(w, op, lane);
        if (lane < nw) s_warp[lane] = wi;  // inclusive over warps
    }
    __syncthreads();
    T before = warp == 0 ? ident : s_warp[warp - 1];
    T excl_in_warp = __shfl_up_sync(0xFFFFFFFFu, inc, 1);
    if (lane == 0) excl_in_warp = ident;
    T res = op(before, excl_in_warp);
    if (total) *total = s_warp[nw - 1];
    __syncthreads();
    return res;
}

struct AddOp {
    template <typename T>
    __device__ T operator()(T a, T b) const { return a + b; }
};
struct MaxOp {
    template <typename T>
    __device__ T operator()(T a, T b) const { return a > b ? a : b; }
};

// ------------------------------------------------------------------ model

// Segment models with the anchors known.  A segment's cone is the
// intersection of its keys' slope intervals (Def. 2 with the anchored Q32
// line), i.e. max (D-eps)/d and min (D+eps+1)/d over its keys; the slope is
// the floor midpoint of the resulting integer interval, and the width is the
// bit length of the largest zigzag residual under that slope (Sec. II-A).
//
// fit_short_kernel: one CTA per window of WK keys, keys staged in shared memory
// (plus kShortMax keys of right halo), one thread per 32-key block: the
// thread fits every segment that starts in its block and has at most
// kShortMax keys, two short sequential passes (cone, then residuals), and
// writes its intercept, start, slope and width.  A longer segment takes the
// slope its chain walk recorded; its widths pass is queued as pieces of
// kPiece keys (long_width_kernel) and its entry is finished by bitoff_kernel.
template <typename KT, uint32_t WK>
__global__ void __launch_bounds__(Win<WK>::kShortThreads)
fit_short_kernel(const KT* __restrict__ keys, const ChunkDesc* __restrict__ chunks, const WinDesc* __restrict__ wins,
                 const uint32_t* __restrict__ tbits, const uint64_t* __restrict__ csb,
                 const LongInfo* __restrict__ longinfo, KT* __restrict__ icpt, int64_t* __restrict__ slope,
                 uint32_t* __restrict__ bitoff, uint16_t* __restrict__ start, uint8_t* __restrict__ width,
                 LongItem* __restrict__ items, uint32_t* __restrict__ nitems, uint32_t items_cap,
                 Piece* __restrict__ pieces, uint32_t* __restrict__ npieces, uint32_t pieces_cap,
                 ulonglong2* __restrict__ cones, uint32_t* __restrict__ status, const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0) return;  // a batch replay that does not fit its plan
    constexpr int kShortThreads = Win<WK>::kShortThreads;
    constexpr uint32_t kLongPerWin = Win<WK>::kLongPerWin;
    extern __shared__ __align__(16) uint8_t smem[];
    constexpr uint32_t kWords = WK / kFB;
    __shared__ uint32_t s_T[kWords + 4];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_base, s_nlong, s_item0, s_piece0;
    // the passes' prefix pieces, then (after a barrier) the window's long segments
    __shared__ union {
        struct {
            ulonglong2 pc[kShortThreads];  // partial cones (pass 1), then largest residuals (pass 2)
            uint32_t pa[kShortThreads];    // their segment's anchor (kNone: none)
        } pieces;
        WinLong lng[kLongPerWin];
    } s_u;
    WinLong* const s_long = s_u.lng;
    const WinDesc wd = wins[blockIdx.x];
    const ChunkDesc cd = chunks[wd.chunk];
    const KT* __restrict__ K = keys + cd.key_begin;
    const uint32_t n = cd.n, w0 = wd.off, w1 = min(n, w0 + WK);
    const int64_t eps = cd.eps;
    const uint32_t tid = threadIdx.x;
    const uint32_t top = min(n, w1 + kShortMax);
    // the low 32 bits of K[i] - K[w0]: a difference of two staged values is
    // exact whenever the true difference is below 2^32, which holds for every
    // run a narrow warp walks; wide warps read their keys from global memory
    uint32_t* s = (uint32_t*)smem;
    const uint64_t kbase = (uint64_t)__ldg(K + w0);
    for (uint32_t q = tid; q < top - w0; q += kShortThreads)
        s[q + (q >> 5)] = (uint32_t)((uint64_t)__ldg(K + w0 + q) - kbase);
    const uint32_t* __restrict__ T = tbits + cd.bitword_begin;
    const uint32_t k0 = w0 / kFB, nT = (top - w0 + kFB - 1) / kFB;
    for (uint32_t q = tid; q < kWords + 4; q += kShortThreads) s_T[q] = q < nT ? T[k0 + q] : 0u;
    // anchors of the chunk before this window
    uint32_t before = 0;
    for (uint32_t q = tid; q < k0; q += kShortThreads) before += __popc(T[q]);
    before = __reduce_add_sync(0xFFFFFFFFu, before);
    if ((tid & 31u) == 0) s_warp[tid >> 5] = before;
    if (tid == 0) s_nlong = 0;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kShortThreads / 32; ++w) t += s_warp[w];
        s_base = t;
    }
    __syncthreads();
    const Staged<uint32_t> st32{s, w0};
    const uint32_t nw = (w1 - w0 + kFB - 1) / kFB;
    const uint32_t word = tid < nw ? s_T[tid] : 0u;
    const uint32_t pre = block_excl_scan<uint32_t>(__popc(word), AddOp(), 0u, s_warp, nullptr);
    uint64_t j = csb[wd.chunk] + s_base + pre;
    const uint64_t* __restrict__ magic = g_magic;
    // the next anchor among the kShortMax = 96 keys after a (bit t: key a + 1 + t), n if the chunk ends
    // first, kNone if neither
    auto next_anchor = [&](uint32_t a) -> uint32_t {
        const uint32_t q = a + 1 - w0, qi = q >> 5, sh = q & 31u;
        const uint64_t lo64 = ((uint64_t)s_T[qi + 1] << 32) | s_T[qi];
        const uint64_t hi64 = ((uint64_t)s_T[qi + 3] << 32) | s_T[qi + 2];
        uint64_t nlo = sh ? (lo64 >> sh) | (hi64 << (64u - sh)) : lo64;  // t = 0..63
        uint32_t nhi = (uint32_t)(hi64 >> sh);                            // t = 64..95
        const uint32_t left = n - a - 1;  // keys after a in the chunk
        if (left < 64) {
            nlo &= (1ull << left) - 1;
            nhi = 0;
        } else if (left < 96) {
            nhi &= (1u << (left - 64)) - 1u;
        }
        if (nlo) return a + 1 + (uint32_t)(__ffsll((long long)nlo) - 1);
        if (nhi) return a + 65 + (uint32_t)(__ffs(nhi) - 1);
        return left < kShortMax ? n : kNone;
    };
    auto is_anchor = [&](uint32_t i) { return (s_T[(i - w0) >> 5] >> ((i - w0) & 31u)) & 1u; };
    // Work is split by keys, not by segments: thread t takes the keys of its
    // 32-key block b (b0 <= i < b1) whatever segment they belong to, so every
    // thread walks about 32 keys.  Its segments are those whose anchor lies in
    // b: all but the last end inside b (the next anchor is in b); the last
    // ends at e_last = next_anchor(a_last) and is short iff that is within 96
    // keys.  The keys of b before its first anchor (the prefix piece) belong
    // to the segment P of the last anchor aP before b0; when P is short and
    // starts in this window, the thread narrows P's cone over them and leaves
    // the partial cone in shared memory, where P's owner merges it (the cone
    // is a max of lower and a min of upper fractions over the keys, so pieces
    // merge exactly).  Keys past the window (at most 95, of the window's last
    // segment) are walked by that segment's owner.
    const uint32_t b0 = w0 + tid * kFB, b1 = min(b0 + kFB, w1);
    const bool has_block = tid < nw;
    uint32_t a_first = 0, a_last = 0, e_last = kNone;
    if (word) {
        a_first = b0 + (uint32_t)(__ffs(word) - 1);
        a_last = b0 + 31u - (uint32_t)__clz(word);
        e_last = next_anchor(a_last);
    }
    uint32_t aP = kNone;  // P's anchor, or kNone: no prefix piece to walk
    if (has_block && !(word & 1u)) {
        for (uint32_t back = 1; back <= 3 && back <= tid && aP == kNone; ++back) {
            const uint32_t wb = s_T[tid - back];
            if (wb) aP = w0 + (tid - back) * kFB + 31u - (uint32_t)__clz(wb);
        }
        if (aP != kNone && next_anchor(aP) == kNone) aP = kNone;  // P is long: its own walk
    }
    const bool tail = word && e_last != kNone && e_last > b1;  // the last segment runs past the block
    const uint32_t pend = word ? a_first : b1;                  // end of the prefix piece
    const uint32_t lo = aP != kNone ? aP : (word ? a_first : b1);
    // the block's keys to walk: up to a long last segment's anchor, else to b1
    const uint32_t wend = word && e_last == kNone ? a_last + 1 : (has_block ? b1 : lo);
    const uint32_t wstart = aP != kNone ? b0 : lo + 1;  // first key walked
    const uint32_t hi = tail ? e_last : wend;            // past the last key any piece of this thread's cones holds
    const uint64_t range = hi > lo + 1 ? (uint64_t)__ldg(K + hi - 1) - (uint64_t)__ldg(K + lo) : 0;
    const bool narrow = __all_sync(0xFFFFFFFFu, range + (uint64_t)eps + 1 < (1ull << 31));
    // key i: its staged offset (narrow warps) or the key itself; the
    // difference of two keys of one walked run, exact either way
    auto key = [&](uint32_t i) -> uint64_t { return narrow ? st32(i) : (uint64_t)__ldg(K + i); };
    auto diff = [&](uint64_t ki, uint64_t kj) -> int64_t {
        return narrow ? (int64_t)(uint32_t)(ki - kj) : (int64_t)(ki - kj);
    };
    const uint64_t j_first = j;
    const uint32_t nown = __popc(word);                           // segments owned, the last maybe long
    const uint32_t nshort = nown - (word && e_last == kNone ? 1u : 0u);
    ulonglong2* const s_pc = s_u.pieces.pc;
    uint32_t* const s_pa = s_u.pieces.pa;
    uint32_t* const s_pz = (uint32_t*)s_u.pieces.pc;  // reused once pass 1's merges are done

    // cone state of the piece being walked
    Frac c = frac_open();
    Frac32 c32 = frac32_open();
    auto cone_key = [&](uint64_t Ki, uint64_t ka, uint32_t d) {
        if (narrow) {
            const uint32_t D = (uint32_t)(Ki - ka);
            const int32_t xl = (int32_t)D - (int32_t)eps;
            const uint32_t yh = D + (uint32_t)eps + 1u;
            if ((int64_t)xl * c32.E > (int64_t)c32.X * d) { c32.X = xl; c32.E = d; }
            if ((uint64_t)yh * c32.F < (uint64_t)c32.Y * d) { c32.Y = yh; c32.F = d; }
        } else {
            const uint64_t D = Ki - ka;
            const int64_t xl = (int64_t)D - eps;
            const uint64_t yh = D + (uint64_t)eps + 1;
            if (frac_gt(xl, d, c.X, c.E)) { c.X = xl; c.E = d; }
            if (yh * (uint64_t)c.F < c.Y * (uint64_t)d) { c.Y = yh; c.F = d; }
        }
    };
    // a cone packed in 16 bytes: E, F <= 95 and |X|, Y < 2^47; E = 0 marks one key
    auto pack = [&](uint32_t nkeys) {
        Frac f = c;
        if (narrow) f = Frac{(int64_t)c32.X, c32.E, (uint64_t)c32.Y, c32.F};
        const uint32_t E = nkeys >= 2 ? f.E : 0u;
        return make_ulonglong2(((uint64_t)f.X & ((1ull << 48) - 1)) | ((uint64_t)E << 48) | ((uint64_t)f.F << 56),
                               f.Y);
    };
    auto reset = [&]() {
        c = frac_open();
        c32 = frac32_open();
    };

    // pass 1: cones.  A closed cone goes to scratch; its slope is taken in
    // pass S, so that no lane waits on another lane's divisions here.
    s_pa[tid] = kNone;
    {
        uint32_t a = lo;
        uint64_t ka = lo < hi ? key(lo) : 0;
        for (uint32_t i = wstart; i < wend; ++i) {
            const uint64_t Ki = key(i);
            if (is_anchor(i)) {
                if (a == aP && i == pend) {  // the prefix piece ends at the block's first anchor
                    s_pc[tid] = pack(2);
                    s_pa[tid] = aP;
                } else {
                    cones[j] = pack(i - a);
                    icpt[j] = __ldg(K + a);
                    start[j] = (uint16_t)a;
                    ++j;
                }
                a = i;
                ka = Ki;
                reset();
                continue;
            }
            cone_key(Ki, ka, i - a);
        }
        if (aP != kNone && !word) {  // the whole block is prefix piece
            s_pc[tid] = pack(2);
            s_pa[tid] = aP;
        } else if (word && e_last != kNone && !tail) {  // the last segment ends at b1
            cones[j] = pack(e_last - a);
            icpt[j] = __ldg(K + a);
            start[j] = (uint16_t)a;
        }
        __syncthreads();
        if (tail) {
            // merge the following blocks' prefix pieces of this segment, then
            // walk its keys past the window
            for (uint32_t u = tid + 1; u < min(tid + 4u, nw) && s_pa[u] == a_last; ++u) {
                const ulonglong2 p = s_pc[u];
                const int64_t X = (int64_t)(p.x << 16) >> 16;
                const uint32_t E = (uint32_t)(p.x >> 48) & 0xFFu, F = (uint32_t)(p.x >> 56);
                if (narrow) {
                    if (X * (int64_t)c32.E > (int64_t)c32.X * (int64_t)E) { c32.X = (int32_t)X; c32.E = E; }
                    if (p.y * (uint64_t)c32.F < (uint64_t)c32.Y * F) { c32.Y = (uint32_t)p.y; c32.F = F; }
                } else {
                    if (frac_gt(X, E, c.X, c.E)) { c.X = X; c.E = E; }
                    if (p.y * (uint64_t)c.F < c.Y * (uint64_t)F) { c.Y = p.y; c.F = F; }
                }
            }
            for (uint32_t i = max(w1, wend); i < e_last; ++i) cone_key(key(i), ka, i - a);
            cones[j] = pack(e_last - a);
            icpt[j] = __ldg(K + a);
            start[j] = (uint16_t)a;
        }
    }
    // pass S: the slope of every owned short segment (floor midpoint, 0 for one key)
    for (uint64_t q = j_first; q < j_first + nshort; ++q) {
        const ulonglong2 cc = cones[q];
        const uint32_t E = (uint32_t)(cc.x >> 48) & 0xFFu;
        int64_t M = 0;
        if (E) {
            Frac f;
            f.X = (int64_t)(cc.x << 16) >> 16;  // sign-extend the 48-bit numerator
            f.E = E;
            f.F = (uint32_t)(cc.x >> 56);
            f.Y = cc.y;
            M = frac_slope(f, magic);
        }
        slope[q] = M;
    }
    __syncthreads();  // P's slope, written by its owner, is read below
    // pass 2: widths, walked the same way
    {
        j = j_first;
        uint32_t a = lo;
        uint64_t ka = lo < hi ? key(lo) : 0;
        int64_t M = aP != kNone ? slope[j_first - 1] : (word ? slope[j_first] : 0);
        uint32_t zmax = 0;
        for (uint32_t i = wstart; i < wend; ++i) {
            const uint64_t Ki = key(i);
            if (is_anchor(i)) {
                if (a == aP && i == pend) {
                    s_pz[tid] = zmax;
                } else {
                    width[j] = (uint8_t)(32u - __clz(zmax));
                    ++j;
                }
                a = i;
                ka = Ki;
                M = j < j_first + nshort ? slope[j] : 0;
                zmax = 0;
                continue;
            }
            zmax = max(zmax, zigzag32(diff(Ki, ka) - line_at(M, i - a)));
        }
        if (aP != kNone && !word) {
            s_pz[tid] = zmax;
        } else if (word && e_last != kNone && !tail) {
            width[j] = (uint8_t)(32u - __clz(zmax));
        }
        __syncthreads();
        if (tail) {
            for (uint32_t u = tid + 1; u < min(tid + 4u, nw) && s_pa[u] == a_last; ++u) zmax = max(zmax, s_pz[u]);
            for (uint32_t i = max(w1, wend); i < e_last; ++i)
                zmax = max(zmax, zigzag32(diff(key(i), ka) - line_at(M, i - a)));
            width[j] = (uint8_t)(32u - __clz(zmax));
        }
    }
    j = j_first + nown - 1;  // the last owned segment (used below when it is long)
    __syncthreads();         // the pieces' storage becomes the long-segment list
    if (word && e_last == kNone) {
        // the segment at a_last is longer than 96 keys: its slope came from the chain's walk
        const uint32_t a = a_last;
        icpt[j] = __ldg(K + a);
        start[j] = (uint16_t)a;
        const LongInfo li = longinfo[cd.bitword_begin + (a >> 5)];
        slope[j] = 0;
        width[j] = 0;
        if (li.end <= a + kShortMax || li.end > n) {  // no walk recorded it: cannot happen
            atomicOr(status, kStInternal);
        } else {
            const uint32_t q = atomicAdd(&s_nlong, 1u);  // at most one per 97 keys: fits
            if (q < kLongPerWin) s_long[q] = WinLong{j, li.M, a, li.end - a};
        }
    }
    // the window's long segments: one reservation of items and pieces for the CTA
    __syncthreads();
    const uint32_t nl = min(s_nlong, kLongPerWin);
    if (tid == 0) {
        uint32_t np = 0;
        for (uint32_t q = 0; q < nl; ++q) {
            s_long[q].poff = np;
            np += (s_long[q].len - 1 + kPiece - 1) / kPiece;
        }
        uint32_t i0 = 0, p0 = 0;
        if (nl) {
            i0 = atomicAdd(nitems, nl);
            p0 = atomicAdd(npieces, np);
        }
        const bool fits = s_nlong <= kLongPerWin && i0 + nl <= items_cap && p0 + np <= pieces_cap;
        if (!fits) atomicOr(status, kStInternal);  // beyond the proven bounds: cannot happen
        s_item0 = i0;
        s_piece0 = p0;
        s_nlong = fits ? nl : 0u;
    }
    __syncthreads();
    for (uint32_t q = tid; q < s_nlong; q += kShortThreads) {
        const WinLong e = s_long[q];
        const uint32_t it = s_item0 + q;
        items[it] = LongItem{cd.key_begin + e.a, e.M, e.len, 0u, 0ull};
        const uint32_t np = (e.len - 1 + kPiece - 1) / kPiece;
        for (uint32_t p = 0; p < np; ++p)
            pieces[s_piece0 + e.poff + p] = Piece{it, 1 + p * kPiece, min(e.len, 1 + (p + 1) * kPiece), 0u};
        slope[e.j] = e.M;
        width[e.j] = 0xFF;  // finished by bitoff_kernel
        bitoff[e.j] = it;
    }
}

// The widths pass of the long segments: one warp per piece of kPiece keys,
// the piece's largest zigzag residual folded into its segment's zmax.
// Pieces are zeroed before fit_short_kernel runs, so a slot that a failed
// (and flagged) reservation left unwritten reads as an empty piece.
template <typename KT>
__global__ void __launch_bounds__(256)
long_width_kernel(const KT* __restrict__ keys, LongItem* __restrict__ items, const Piece* __restrict__ pieces,
                  const uint32_t* __restrict__ npieces, uint32_t pieces_cap, const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0) return;
    const uint32_t np = min(*npieces, pieces_cap);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < np; p += nwarps) {
        const Piece pc = pieces[p];
        if (pc.t0 >= pc.t1) continue;
        const LongItem it = items[pc.item];
        const KT* __restrict__ K = keys + it.key0;
        const uint64_t ka = ldk(K, 0);
        uint32_t z = 0;
        uint32_t t = pc.t0 + lane;
        for (; t + 96 < pc.t1; t += 128) {
            const uint64_t k0 = ldk(K, t), k1 = ldk(K, t + 32), k2 = ldk(K, t + 64), k3 = ldk(K, t + 96);
            z = max(z, zigzag32((int64_t)(k0 - ka) - line_at(it.M, t)));
            z = max(z, zigzag32((int64_t)(k1 - ka) - line_at(it.M, t + 32)));
            z = max(z, zigzag32((int64_t)(k2 - ka) - line_at(it.M, t + 64)));
            z = max(z, zigzag32((int64_t)(k3 - ka) - line_at(it.M, t + 96)));
        }
        for (; t < pc.t1; t += 32) z = max(z, zigzag32((int64_t)(ldk(K, t) - ka) - line_at(it.M, t)));
        z = __reduce_max_sync(0xFFFFFFFFu, z);
        if (lane == 0 && z) atomicMax(&items[pc.item].zmax, z);
    }
}

// One CTA per chunk: the long segments' widths, then the bit offsets of the
// chunk's segments in order (a scan of w (n - 1)), and the chunk's bit count.
__global__ void __launch_bounds__(256)
bitoff_kernel(const ChunkDesc* __restrict__ chunks, const uint64_t* __restrict__ csb,
              const LongItem* __restrict__ items, uint32_t* __restrict__ bitoff, const uint16_t* __restrict__ start,
              uint8_t* __restrict__ width, uint32_t* __restrict__ chunk_bits, const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ uint32_t s_scan[32];
    const uint32_t n = chunks[blockIdx.x].n;
    const uint64_t s0 = csb[blockIdx.x], s1 = csb[blockIdx.x + 1];
    uint32_t carry = 0;
    for (uint64_t b0 = s0; b0 < s1; b0 += blockDim.x) {
        const uint64_t j = b0 + threadIdx.x;
        uint32_t bits = 0;
        if (j < s1) {
            uint32_t w = width[j];
            if (w == 0xFF) {
                w = 32u - __clz(items[bitoff[j]].zmax);
                width[j] = (uint8_t)w;
            }
            const uint32_t st = start[j];
            const uint32_t en = j + 1 < s1 ? (uint32_t)start[j + 1] : n;
            bits = w * (en - st - 1);
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan<uint32_t>(bits, AddOp(), 0u, s_scan, &tot);
        if (j < s1) bitoff[j] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) chunk_bits[blockIdx.x] = carry;
}

// ------------------------------------------------------------------ pack

template <typename KT>
__global__ void __launch_bounds__(kPackThreads)
pack_kernel(const KT* __restrict__ keys, const ChunkDesc* __restrict__ chunks, const uint32_t* __restrict__ tbits,
            const uint64_t* __restrict__ csb, const uint64_t* __restrict__ cwb, const KT* __restrict__ icpt,
            const int64_t* __restrict__ slope, const uint32_t* __restrict__ bitoff,
            const uint16_t* __restrict__ start, const uint8_t* __restrict__ width, uint32_t* __restrict__ pay32,
            const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ uint32_t s_T[kMaxChunk / 32];
    __shared__ uint32_t s_pref[kMaxChunk / 32];
    __shared__ uint32_t s_buf[kWin + 4];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_end_bit;

    const ChunkDesc cd = chunks[blockIdx.x];
    const KT* __restrict__ K = keys + cd.key_begin;
    const uint32_t n = cd.n;
    const uint32_t tid = threadIdx.x;
    const uint32_t nwords = (n + 31) / 32;
    // per-word exclusive popcount prefix of the anchor bitmap (8 words per thread)
    uint32_t loc[8];
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint32_t wd = tid * 8 + q;
        const uint32_t v = wd < nwords ? tbits[cd.bitword_begin + wd] : 0u;
        loc[q] = v;
        sum += __popc(v);
    }
    uint32_t run = block_excl_scan<uint32_t>(sum, AddOp(), 0u, s_warp, nullptr);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint32_t wd = tid * 8 + q;
        if (wd < nwords) {
            s_T[wd] = loc[q];
            s_pref[wd] = run;
        }
        run += __popc(loc[q]);
    }
    __syncthreads();

    const uint64_t seg0 = csb[blockIdx.x];
    const uint64_t pbase = 2 * cwb[blockIdx.x];                       // chunk payload, 32-bit words
    const uint64_t pwords = 2 * (cwb[blockIdx.x + 1] - cwb[blockIdx.x]);
    uint32_t cur_bit = 0;  // bits of the chunk payload already final
    uint32_t carry = 0;    // bits [32*(cur_bit>>5), cur_bit) of the next word
    for (uint32_t w0 = 0; w0 < n; w0 += kWin) {
        const uint32_t w1 = min(n, w0 + kWin);
        const uint32_t base_word = cur_bit >> 5;
        for (uint32_t q = tid; q < kWin + 4; q += kPackThreads) s_buf[q] = 0;
        if (tid == 0) s_buf[0] = carry;
        __syncthreads();
        if (tid == 0) {
            // end of the window's bits: the last key's residual end
            const uint32_t i = w1 - 1;
            const uint32_t wd = i >> 5;
            const uint32_t r = s_pref[wd] + __popc(s_T[wd] & (0xFFFFFFFFu >> (31u - (i & 31u)))) - 1;
            const uint64_t j = seg0 + r;
            const uint32_t a = start[j];
            s_end_bit = bitoff[j] + (uint32_t)width[j] * (i - a);
        }
        for (uint32_t i = w0 + tid; i < w1; i += kPackThreads) {
            const uint32_t wd = i >> 5;
            const uint32_t tw = s_T[wd];
            if ((tw >> (i & 31u)) & 1u) continue;  // anchors store no residual
            const uint32_t r = s_pref[wd] + __popc(tw & (0xFFFFFFFFu >> (31u - (i & 31u)))) - 1;
            const uint64_t j = seg0 + r;
            const uint32_t a = __ldg(start + j);
            const uint32_t w = __ldg(width + j);
            if (w == 0) continue;
            const uint32_t d = i - a;
            const uint64_t D = ldk(K, i) - (uint64_t)__ldg(icpt + j);
            const int64_t res = (int64_t)D - line_at(__ldg(slope + j), d);
            const uint32_t z = zigzag32(res);
            const uint32_t pos = __ldg(bitoff + j) + w * (d - 1) - 32u * base_word;
            const uint32_t sh = pos & 31u;
            atomicOr(&s_buf[pos >> 5], z << sh);
            if (sh + w > 32) atomicOr(&s_buf[(pos >> 5) + 1], z >> (32u - sh));
        }
        __syncthreads();
        const uint32_t end_bit = s_end_bit;
        const uint32_t full = (end_bit >> 5) - base_word;  // words now final
        for (uint32_t q = tid; q < full; q += kPackThreads) pay32[pbase + base_word + q] = s_buf[q];
        carry = s_buf[full];
        cur_bit = end_bit;
        __syncthreads();
    }
    // the partial last word, then the zero padding to the chunk's even word count
    const uint32_t first = cur_bit >> 5;
    for (uint64_t q = first + tid; q < pwords; q += kPackThreads) pay32[pbase + q] = (q == first) ? carry : 0u;
}

// ------------------------------------------------------------------ device-wide exclusive scan


__device__ __forceinline__ uint64_t scan_val(uint32_t v, ScanOp op) {
    if (op == ScanOp::Identity) return v;
    const uint64_t w = ((uint64_t)v + 63) / 64;
    return w + (w & 1);
}

__global__ void scan_reduce(const uint32_t* __restrict__ in, uint64_t n, ScanOp op, uint64_t* __restrict__ part) {
    __shared__ uint64_t s_warp[32];
    const uint64_t base = blockIdx.x * kScanTile;
    uint64_t s = 0;
    for (int q = 0; q < kScanItems; ++q) {
        const uint64_t i = base + (uint64_t)threadIdx.x * kScanItems + q;
        if (i < n) s += scan_val(in[i], op);
    }
    uint64_t tot;
    block_excl_scan<uint64_t>(s, AddOp(), 0ull, s_warp, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void scan_parts(uint64_t* __restrict__ part, uint64_t nparts) {
    __shared__ uint64_t s_warp[32];
    __shared__ uint64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint64_t b = 0; b < nparts; b += blockDim.x) {
        const uint64_t i = b + threadIdx.x;
        const uint64_t v = i < nparts ? part[i] : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_scan<uint64_t>(v, AddOp(), 0ull, s_warp, &tot);
        if (i < nparts) part[i] = s_carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
    }
}

__global__ void scan_final(const uint32_t* __restrict__ in, uint64_t n, ScanOp op, const uint64_t* __restrict__ part,
                           uint64_t* __restrict__ out) {
    __shared__ uint64_t s_warp[32];
    const uint64_t base = blockIdx.x * kScanTile;
    uint64_t v[kScanItems];
    uint64_t s = 0;
    for (int q = 0; q < kScanItems; ++q) {
        const uint64_t i = base + (uint64_t)threadIdx.x * kScanItems + q;
        v[q] = i < n ? scan_val(in[i], op) : 0;
        s += v[q];
    }
    uint64_t tot;
    uint64_t run = part[blockIdx.x] + block_excl_scan<uint64_t>(s, AddOp(), 0ull, s_warp, &tot);
    for (int q = 0; q < kScanItems; ++q) {
        const uint64_t i = base + (uint64_t)threadIdx.x * kScanItems + q;
        if (i < n) out[i] = run;
        run += v[q];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = part[blockIdx.x] + tot;
}

}  // namespace

size_t scan_tmp_bytes(uint64_t n) { return sizeof(uint64_t) * ((n + kScanTile - 1) / kScanTile + 1); }

int scan_exclusive(const uint32_t* in, uint64_t* out, uint64_t n, ScanOp op, void* tmp, size_t tmp_bytes,
                   cudaStream_t st) {
    if (n == 0) return cuda_status(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
    const uint64_t nb = (n + kScanTile - 1) / kScanTile;
    if (tmp_bytes < nb * sizeof(uint64_t)) return LC_ERR_INTERNAL;
    uint64_t* part = (uint64_t*)tmp;
    {
        KTime kt("scan", st);
        scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, op, part);
        scan_parts<<<1, kScanThreads, 0, st>>>(part, nb);
        scan_final<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, op, part, out);
    }
    note_launch(3);
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ host pipeline

static int ensure_magic() {
    static DeviceOnce once;
    return once_per_device(once, [] {
        std::vector<uint64_t> m(kMaxChunk, 0);
        for (uint32_t d = 2; d < kMaxChunk; ++d) {
            const unsigned __int128 two64 = (unsigned __int128)1 << 64;
            m[d] = (uint64_t)((two64 + d - 1) / d);
        }
        return cuda_status(cudaMemcpyToSymbol(g_magic, m.data(), m.size() * sizeof(uint64_t)));
    });
}

// Keys covered by the chunk table (the reach array is indexed like the keys).
static uint64_t nkeys_total_of(const ChunkDesc* ch, uint64_t C) {
    return C ? ch[C - 1].key_begin + ch[C - 1].n : 0;
}

static int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

struct FitScratch {
    const WinDesc* wins;
    uint64_t nwins;
    uint32_t span_log2;  // keys per speculating thread: 2^5, 2^6 (default) or 2^7
    uint32_t win_keys;   // keys per window: kWinWide or kWinNarrow
    uint32_t *spec, *entry, *exit;
    LongInfo* longinfo;
    LongItem* items;
    Piece* pieces;
    uint32_t* counters;  // [0] long items, [1] pieces
    ulonglong2* cones;   // stage 1: the cone of every short segment [L]
    uint8_t* roff;       // jump fit: reach of every key [N] (nullptr: greedy only)
    uint32_t* jbits;     // jump fit: anchor bits [bitwords]
    LongInfo* jlong;     // jump fit: long-segment records [bitwords]
    uint32_t items_cap, pieces_cap;
};

// The window size of a run: narrow windows for chunks of a few thousand keys
// on average (columns of short lists), where a wide window would leave most
// of its threads idle; wide ones otherwise, and always at a span of 128 keys
// (a narrow window would then give the speculation a CTA of 16 threads).
static uint32_t window_keys(uint64_t nkeys, uint64_t C, uint32_t span_log2) {
    if (span_log2 == 7 || C == 0) return kWinWide;
    return nkeys / C < 4 * (uint64_t)kWinWide ? kWinNarrow : kWinWide;
}

// The speculative walks (stage 0), the short models (stage 1) or the jump
// fit's reach per key (stage 2) for one window size.
template <typename KT, uint32_t WK>
static int run_windows(const KT* keys, const ChunkDesc* chunks_d, const FitScratch& fs, uint32_t* tbits,
                       uint32_t* status, uint8_t* blob, const Layout& lay, cudaStream_t st, int stage,
                       const uint32_t* gate) {
    using Wn = Win<WK>;
    if (stage == 0) {
        const size_t smem = sizeof(uint32_t) * Wn::kSpecSlots;
        static DeviceOnce once1, once2, once4;
        int rc = LC_OK;
        KTime kt("fit_spec", st);
        if (fs.span_log2 == 5) {
            if (!(rc = smem_attr_once(once1, spec_kernel<KT, 1, WK>, smem)))
                spec_kernel<KT, 1, WK><<<(unsigned)fs.nwins, WK / 32, smem, st>>>(keys, chunks_d, fs.wins, fs.spec,
                                                                                  fs.entry, fs.exit, status);
        } else if (fs.span_log2 == 7) {
            if constexpr (WK / 128 >= 32) {
                if (!(rc = smem_attr_once(once4, spec_kernel<KT, 4, WK>, smem)))
                    spec_kernel<KT, 4, WK><<<(unsigned)fs.nwins, WK / 128, smem, st>>>(keys, chunks_d, fs.wins,
                                                                                       fs.spec, fs.entry, fs.exit,
                                                                                       status);
            } else {
                rc = LC_ERR_INTERNAL;  // window_keys never pairs this span with a narrow window
            }
        } else {
            if (!(rc = smem_attr_once(once2, spec_kernel<KT, 2, WK>, smem)))
                spec_kernel<KT, 2, WK><<<(unsigned)fs.nwins, WK / 64, smem, st>>>(keys, chunks_d, fs.wins, fs.spec,
                                                                                  fs.entry, fs.exit, status);
        }
        return rc;
    }
    if (stage == 2) {
        static DeviceOnce once_r;
        const size_t rsm = sizeof(uint32_t) * Wn::kShortSlots;
        if (int rc = smem_attr_once(once_r, reach_kernel<KT, WK>, rsm)) return rc;
        KTime kt("jump_reach", st);
        reach_kernel<KT, WK><<<(unsigned)fs.nwins, Wn::kShortThreads, rsm, st>>>(keys, chunks_d, fs.wins, fs.roff);
        return LC_OK;
    }
    static DeviceOnce once_s;
    const size_t smem = sizeof(uint32_t) * Wn::kShortSlots;
    if (int rc = smem_attr_once(once_s, fit_short_kernel<KT, WK>, smem)) return rc;
    KTime kt("model_short", st);
    fit_short_kernel<KT, WK><<<(unsigned)fs.nwins, Wn::kShortThreads, smem, st>>>(
        keys, chunks_d, fs.wins, tbits, (const uint64_t*)(blob + lay.csb), fs.longinfo, (KT*)(blob + lay.icpt),
        (int64_t*)(blob + lay.slope), (uint32_t*)(blob + lay.bitoff), (uint16_t*)(blob + lay.start),
        (uint8_t*)(blob + lay.width), fs.items, fs.counters, fs.items_cap, fs.pieces, fs.counters + 1,
        fs.pieces_cap, fs.cones, status, gate);
    return LC_OK;
}

template <typename KT>
static int run_windows(const KT* keys, const ChunkDesc* chunks_d, const FitScratch& fs, uint32_t* tbits,
                       uint32_t* status, uint8_t* blob, const Layout& lay, cudaStream_t st, int stage,
                       const uint32_t* gate) {
    return fs.win_keys == kWinNarrow
               ? run_windows<KT, kWinNarrow>(keys, chunks_d, fs, tbits, status, blob, lay, st, stage, gate)
               : run_windows<KT, kWinWide>(keys, chunks_d, fs, tbits, status, blob, lay, st, stage, gate);
}

template <typename KT>
static int run_pipeline(const KT* keys, const ChunkDesc* chunks_d, uint64_t C, const FitScratch& fs, uint32_t* tbits,
                        uint32_t* counts, uint64_t* csb, uint32_t* status, void* tmp, size_t tmp_bytes,
                        lc_column* col, cudaStream_t st, int stage, const uint32_t* gate = nullptr) {
    uint8_t* blob = col->blob;
    const Layout& lay = col->lay;
    if (stage == 0) {
        int rc = run_windows<KT>(keys, chunks_d, fs, tbits, status, blob, lay, st, 0, gate);
        if (rc) return rc;
        {
            KTime kt("fit_chain", st);
            chain_kernel<KT><<<(unsigned)((C + kChainThreads / 32 - 1) / (kChainThreads / 32)), kChainThreads, 0, st>>>(
                keys, chunks_d, C, fs.spec, fs.entry, fs.exit, tbits, counts, fs.longinfo);
        }
        note_launch(2);
        rc = cuda_status(cudaGetLastError());
        if (rc) return rc;
        if (fs.roff) {
            if ((rc = run_windows<KT>(keys, chunks_d, fs, tbits, status, blob, lay, st, 2, gate))) return rc;
            {
                KTime kt("jump_chain", st);
                jump_kernel<KT><<<(unsigned)((C + kChainThreads / 32 - 1) / (kChainThreads / 32)), kChainThreads, 0,
                                  st>>>(keys, chunks_d, C, fs.roff, tbits, counts, fs.longinfo, fs.jbits, fs.jlong);
            }
            note_launch(2);
            rc = cuda_status(cudaGetLastError());
            if (rc) return rc;
        }
        return scan_exclusive(counts, csb, C, ScanOp::Identity, tmp, tmp_bytes, st);
    }
    if (int rc = run_windows<KT>(keys, chunks_d, fs, tbits, status, blob, lay, st, 1, gate)) return rc;
    {
        KTime kt("model_long", st);
        long_width_kernel<KT><<<(unsigned)(device_sms() * 8), 256, 0, st>>>(keys, fs.items, fs.pieces, fs.counters + 1,
                                                                          fs.pieces_cap, gate);
    }
    {
        KTime kt("bitoff", st);
        bitoff_kernel<<<(unsigned)C, 256, 0, st>>>(chunks_d, (const uint64_t*)(blob + lay.csb), fs.items,
                                                   (uint32_t*)(blob + lay.bitoff), (const uint16_t*)(blob + lay.start),
                                                   (uint8_t*)(blob + lay.width), counts, gate);
    }
    note_launch(3);
    int rc = cuda_status(cudaGetLastError());
    if (rc) return rc;
    rc = scan_exclusive(counts, (uint64_t*)(blob + lay.cwb), C, ScanOp::BitsToEvenWords, tmp, tmp_bytes, st);
    if (rc) return rc;
    {
        KTime kt("pack", st);
        pack_kernel<KT><<<(unsigned)C, kPackThreads, 0, st>>>(
            keys, chunks_d, tbits, (const uint64_t*)(blob + lay.csb), (const uint64_t*)(blob + lay.cwb),
            (const KT*)(blob + lay.icpt), (const int64_t*)(blob + lay.slope), (const uint32_t*)(blob + lay.bitoff),
            (const uint16_t*)(blob + lay.start), (const uint8_t*)(blob + lay.width), (uint32_t*)(blob + lay.payload),
            gate);
    }
    note_launch();
    return cuda_status(cudaGetLastError());
}

// The compress pipeline's scratch: chunk table, windows, per-block fit state,
// anchor bitmap, per-chunk counts, scan partials, status, chunk_seg_begin,
// long-segment records, their width-pass items and pieces.
struct PipeScratch {
    std::vector<WinDesc> wins;
    uint64_t nwins = 0, C = 0, bitwords = 0, items_cap = 0, pieces_cap = 0;
    uint32_t win_keys = kWinWide, span_log2 = 6;
    size_t off_chunks = 0, off_wins = 0, off_blk = 0, off_bits = 0, off_counts = 0, off_tmp = 0, off_status = 0,
           off_csb = 0, off_long = 0, off_items = 0, off_pieces = 0, off_counters = 0, bytes = 0, tmp_bytes = 0;
    ChunkDesc* chunks_d = nullptr;
    uint32_t *tbits = nullptr, *counts = nullptr, *status = nullptr;
    uint64_t* csb_tmp = nullptr;
    void* tmp = nullptr;

    // Windows and offsets for a chunk table; returns the bytes to allocate.
    size_t plan(const ChunkDesc* chunks_h, uint64_t C_, uint64_t bitwords_, uint32_t span_log2_) {
        C = C_;
        bitwords = bitwords_;
        span_log2 = span_log2_;
        win_keys = window_keys(nkeys_total_of(chunks_h, C), C, span_log2);
        wins.clear();
        for (uint64_t c = 0; c < C; ++c)
            for (uint32_t off = 0; off < chunks_h[c].n; off += win_keys) wins.push_back(WinDesc{(uint32_t)c, off});
        nwins = wins.size();
        tmp_bytes = scan_tmp_bytes(C);
        auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
        off_chunks = 0;
        off_wins = al(off_chunks + C * sizeof(ChunkDesc));
        off_blk = al(off_wins + nwins * sizeof(WinDesc));
        off_bits = al(off_blk + 3 * 4 * bitwords);
        off_counts = al(off_bits + bitwords * 4);
        off_tmp = al(off_counts + (C + 1) * 4);
        off_status = al(off_tmp + tmp_bytes);
        off_csb = al(off_status + 256);
        // long segments (> kShortMax keys): at most one per 32-key block, N / (kShortMax + 1) in all
        uint64_t nkeys = 0;
        for (uint64_t c = 0; c < C; ++c) nkeys += chunks_h[c].n;
        items_cap = std::min<uint64_t>(nkeys / (kShortMax + 1) + 1, 0xFFFFFFFFull);
        pieces_cap = std::min<uint64_t>(items_cap + nkeys / kPiece + 1, 0xFFFFFFFFull);
        off_long = al(off_csb + (C + 1) * sizeof(uint64_t));
        off_items = al(off_long + bitwords * sizeof(LongInfo));
        off_pieces = al(off_items + items_cap * sizeof(LongItem));
        off_counters = al(off_pieces + pieces_cap * sizeof(Piece));
        bytes = off_counters + 256;
        return bytes;
    }
    FitScratch bind(uint8_t* scratch) {
        chunks_d = (ChunkDesc*)(scratch + off_chunks);
        tbits = (uint32_t*)(scratch + off_bits);
        counts = (uint32_t*)(scratch + off_counts);
        tmp = scratch + off_tmp;
        status = (uint32_t*)(scratch + off_status);
        csb_tmp = (uint64_t*)(scratch + off_csb);
        FitScratch fs;
        fs.wins = (const WinDesc*)(scratch + off_wins);
        fs.nwins = nwins;
        fs.spec = (uint32_t*)(scratch + off_blk);
        fs.entry = fs.spec + bitwords;
        fs.exit = fs.entry + bitwords;
        fs.longinfo = (LongInfo*)(scratch + off_long);
        fs.items = (LongItem*)(scratch + off_items);
        fs.pieces = (Piece*)(scratch + off_pieces);
        fs.counters = (uint32_t*)(scratch + off_counters);
        fs.items_cap = (uint32_t)items_cap;
        fs.pieces_cap = (uint32_t)pieces_cap;
        fs.cones = nullptr;
        fs.roff = nullptr;
        fs.jbits = nullptr;
        fs.jlong = nullptr;
        fs.span_log2 = span_log2;
        fs.win_keys = win_keys;
        return fs;
    }
    // The per-run resets the pipeline expects (status, long-segment records, counters, pieces).
    int reset(const FitScratch& fs, cudaStream_t st) const {
        int rc = cuda_status(cudaMemsetAsync(status, 0, 4, st));
        if (!rc) rc = cuda_status(cudaMemsetAsync(fs.longinfo, 0, bitwords * sizeof(LongInfo), st));
        if (!rc) rc = cuda_status(cudaMemsetAsync(fs.counters, 0, 8, st));
        if (!rc) rc = cuda_status(cudaMemsetAsync(fs.pieces, 0, pieces_cap * sizeof(Piece), st));
        return rc;
    }
};

int compress_impl(const void* keys_dev, int kb, const ChunkDesc* chunks_h, uint64_t C, uint64_t bitwords,
                  uint64_t payload_bound_words, cudaStream_t st, lc_column* col, bool jump, uint32_t span_log2) {
    int rc = ensure_magic();
    if (rc) return rc;
    PipeScratch ps;
    uint8_t* scratch = nullptr;
    if (cudaMallocAsync((void**)&scratch, ps.plan(chunks_h, C, bitwords, span_log2), st) != cudaSuccess)
        return LC_ERR_NOMEM;
    FitScratch fs = ps.bind(scratch);
    const std::vector<WinDesc>& wins = ps.wins;
    const uint64_t nwins = ps.nwins;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t off_wins = ps.off_wins;
    ChunkDesc* chunks_d = ps.chunks_d;
    uint32_t* tbits = ps.tbits;
    uint32_t* counts = ps.counts;
    void* tmp = ps.tmp;
    const size_t tmp_bytes = ps.tmp_bytes;
    uint32_t* status = ps.status;
    uint64_t* csb_tmp = ps.csb_tmp;
    uint64_t total = 0;
    uint32_t h_status = 0;
    fs.cones = nullptr;
    fs.roff = nullptr;
    fs.jbits = nullptr;
    fs.jlong = nullptr;
    uint8_t* jscratch = nullptr;
    auto fail = [&](int code) {
        cudaStreamSynchronize(st);
        cudaFreeAsync(scratch, st);
        if (fs.cones) cudaFreeAsync(fs.cones, st);
        if (jscratch) cudaFreeAsync(jscratch, st);
        return code;
    };
    if (jump) {
        // reach per key, anchor bits and long-segment records of the jump segmentation
        const uint64_t o_bits = al(nkeys_total_of(chunks_h, C)), o_long = o_bits + al(4 * bitwords);
        if (cudaMallocAsync((void**)&jscratch, o_long + sizeof(LongInfo) * bitwords + 256, st) != cudaSuccess) {
            jscratch = nullptr;
            return fail(LC_ERR_NOMEM);
        }
        fs.roff = jscratch;
        fs.jbits = (uint32_t*)(jscratch + o_bits);
        fs.jlong = (LongInfo*)(jscratch + o_long);
    }

    rc = stage_h2d(scratch + off_wins, wins.data(), nwins * sizeof(WinDesc), st);
    if (rc) return fail(rc);
    rc = stage_h2d(chunks_d, chunks_h, C * sizeof(ChunkDesc), st);
    if (rc) return fail(rc);
    rc = ps.reset(fs, st);
    if (rc) return fail(rc);

    // stage 0: anchors and segment counts
    HTime ht0("fit_stage0");
    if (kb == 4)
        rc = run_pipeline<uint32_t>((const uint32_t*)keys_dev, chunks_d, C, fs, tbits, counts, csb_tmp, status, tmp,
                                    tmp_bytes, col, st, 0);
    else
        rc = run_pipeline<uint64_t>((const uint64_t*)keys_dev, chunks_d, C, fs, tbits, counts, csb_tmp, status, tmp,
                                    tmp_bytes, col, st, 0);
    if (rc) return fail(rc);
    const void *p_total = nullptr, *p_status = nullptr;
    rc = stage_d2h(csb_tmp + C, 8, st, &p_total);
    if (rc) return fail(rc);
    rc = stage_d2h(status, 4, st, &p_status);
    if (rc) return fail(rc);
    rc = stage_sync(st);
    if (rc) return fail(rc);
    std::memcpy(&total, p_total, 8);
    std::memcpy(&h_status, p_status, 4);
    if (h_status & kStUnsorted) return fail(LC_ERR_UNSORTED);
    const uint64_t L = total;
    HTime ht1("fit_stage1");

    // the blob, with the payload sized by the paper's bound of
    // ceil(log2(2 eps + 1)) bits per residual (plus per-chunk padding)
    Layout lay = make_layout(kb, C, L, payload_bound_words, col->NL, col->list_mode != 0);
    col->L = L;
    col->blob_cap = lay.total;
    if (cudaMallocAsync((void**)&col->blob, lay.total, st) != cudaSuccess) {
        col->blob = nullptr;
        return fail(LC_ERR_NOMEM);
    }
    col->lay = lay;
    rc = cuda_status(cudaMemcpyAsync(col->blob + lay.csb, csb_tmp, (C + 1) * 8, cudaMemcpyDeviceToDevice, st));
    if (rc) return fail(rc);
    // the cones of the short segments between the fit's two passes (16 bytes per segment)
    if (cudaMallocAsync((void**)&fs.cones, 16 * std::max<uint64_t>(L, 1), st) != cudaSuccess) {
        fs.cones = nullptr;
        return fail(LC_ERR_NOMEM);
    }

    // stage 1: model, widths, payload
    if (kb == 4)
        rc = run_pipeline<uint32_t>((const uint32_t*)keys_dev, chunks_d, C, fs, tbits, counts, csb_tmp, status, tmp,
                                    tmp_bytes, col, st, 1);
    else
        rc = run_pipeline<uint64_t>((const uint64_t*)keys_dev, chunks_d, C, fs, tbits, counts, csb_tmp, status, tmp,
                                    tmp_bytes, col, st, 1);
    if (rc) return fail(rc);
    // the derived directories' memory, taken while stage 1 runs: a large
    // stream-ordered allocation costs the host a few hundred microseconds,
    // which would otherwise leave the device idle (build_derived allocates it
    // if this did not)
    if (!col->derived2 &&
        cudaMallocAsync((void**)&col->derived2, derived2_layout(col->N, L, col->list_mode != 0).bytes, st) !=
            cudaSuccess)
        col->derived2 = nullptr;
    rc = stage_d2h(col->blob + lay.cwb + 8 * C, 8, st, &p_total);
    if (rc) return fail(rc);
    rc = stage_d2h(status, 4, st, &p_status);
    if (rc) return fail(rc);
    rc = stage_sync(st);
    if (rc) return fail(rc);
    std::memcpy(&total, p_total, 8);
    std::memcpy(&h_status, p_status, 4);
    if (total > payload_bound_words || (h_status & kStInternal)) return fail(LC_ERR_INTERNAL);
    col->W = total;
    col->lay = make_layout(kb, C, L, col->W, col->NL, col->list_mode != 0);
    cudaFreeAsync(scratch, st);
    cudaFreeAsync(fs.cones, st);
    if (jscratch) cudaFreeAsync(jscratch, st);
    return LC_OK;
}

// ------------------------------------------------------------------ the batching graph

namespace {
// A replay's check against its plan: *gate = 1 while the device total equals
// the planned one (and, after the first check, the gate was open), else 0,
// with kStPlan in the column's status word.
__global__ void plan_gate_kernel(const uint64_t* __restrict__ total, uint64_t want, uint32_t* __restrict__ gate,
                                 uint32_t* __restrict__ status, int first) {
    if (threadIdx.x == 0) {
        const bool ok = *total == want && (first || *gate != 0u);
        *gate = ok ? 1u : 0u;
        if (!ok) atomicOr(status, kStPlan);
    }
}
}  // namespace

struct BatchGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint8_t* scratch = nullptr;  // the pipeline's scratch, the cones, the gate, the derived directories' scan scratch
};

void batch_graph_free(BatchGraph* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->scratch) {
        cudaDeviceSynchronize();
        cudaFree(g->scratch);
    }
    delete g;
}

int batch_graph_launch(BatchGraph* g, cudaStream_t st) { return cuda_status(cudaGraphLaunch(g->exec, st)); }

template <typename KT>
static int batch_enqueue(const KT* keys, const PipeScratch& ps, const FitScratch& fs, lc_column* col, uint32_t* gate,
                         void* dtmp, size_t dtmp_bytes, void* out_dev, cudaStream_t st) {
    const Layout& lay = col->lay;
    int rc = ps.reset(fs, st);
    if (!rc) rc = run_pipeline<KT>(keys, ps.chunks_d, ps.C, fs, ps.tbits, ps.counts, ps.csb_tmp, ps.status, ps.tmp,
                                   ps.tmp_bytes, col, st, 0);
    if (rc) return rc;
    plan_gate_kernel<<<1, 32, 0, st>>>(ps.csb_tmp + ps.C, col->L, gate, col->status, 1);
    note_launch();
    rc = cuda_status(cudaMemcpyAsync(col->blob + lay.csb, ps.csb_tmp, (ps.C + 1) * 8, cudaMemcpyDeviceToDevice, st));
    if (!rc) rc = run_pipeline<KT>(keys, ps.chunks_d, ps.C, fs, ps.tbits, ps.counts, ps.csb_tmp, ps.status, ps.tmp,
                                   ps.tmp_bytes, col, st, 1, gate);
    if (rc) return rc;
    plan_gate_kernel<<<1, 32, 0, st>>>((const uint64_t*)(col->blob + lay.cwb) + ps.C, col->W, gate, col->status, 0);
    note_launch();
    rc = cuda_status(cudaGetLastError());
    if (!rc) rc = derived_replay(col, gate, dtmp, dtmp_bytes, out_dev, st);
    return rc;
}

int batch_graph_build(const void* keys_dev, int kb, const ChunkDesc* chunks_h, uint64_t C, uint64_t bitwords,
                      uint32_t span_log2, lc_column* col, void* out_dev, cudaStream_t st, BatchGraph** out) {
    *out = nullptr;
    if (!col->list_mode || C == 0) return LC_ERR_INVALID_ARG;
    BatchGraph* g = new (std::nothrow) BatchGraph;
    if (!g) return LC_ERR_NOMEM;
    PipeScratch ps;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t pipe = al(ps.plan(chunks_h, C, bitwords, span_log2));
    const size_t off_cones = pipe, off_gate = al(off_cones + 16 * std::max<uint64_t>(col->L, 1));
    const size_t off_dtmp = al(off_gate + 256), dtmp_bytes = derived_replay_tmp_bytes(col);
    int rc = cuda_status(cudaMalloc((void**)&g->scratch, off_dtmp + dtmp_bytes + 256));
    if (rc) {
        g->scratch = nullptr;
        batch_graph_free(g);
        return rc;
    }
    FitScratch fs = ps.bind(g->scratch);
    fs.cones = (ulonglong2*)(g->scratch + off_cones);
    uint32_t* gate = (uint32_t*)(g->scratch + off_gate);
    // the descriptors are uploaded once; the graph reads them on every replay
    rc = stage_h2d(g->scratch + ps.off_wins, ps.wins.data(), ps.nwins * sizeof(WinDesc), st);
    if (!rc) rc = stage_h2d(ps.chunks_d, chunks_h, C * sizeof(ChunkDesc), st);
    if (!rc) rc = stage_sync(st);
    cudaStream_t cs = nullptr;
    if (!rc) rc = cuda_status(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (!rc) rc = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    if (!rc) {
        const int rk = kb == 4 ? batch_enqueue<uint32_t>((const uint32_t*)keys_dev, ps, fs, col, gate,
                                                         g->scratch + off_dtmp, dtmp_bytes, out_dev, cs)
                               : batch_enqueue<uint64_t>((const uint64_t*)keys_dev, ps, fs, col, gate,
                                                         g->scratch + off_dtmp, dtmp_bytes, out_dev, cs);
        const int re = cuda_status(cudaStreamEndCapture(cs, &g->graph));
        rc = rk ? rk : re;
    }
    if (!rc) rc = cuda_status(cudaGraphInstantiate(&g->exec, g->graph, 0));
    if (cs) cudaStreamDestroy(cs);
    if (rc) {
        batch_graph_free(g);
        return rc;
    }
    *out = g;
    return LC_OK;
}

namespace {
struct PadRanges {
    uint64_t r[2 * 16];
    int n;
};
__global__ void zero_pads(uint8_t* __restrict__ p, PadRanges pr) {
    for (int r = 0; r < pr.n; ++r)
        for (uint64_t i = pr.r[2 * r] + threadIdx.x; i < pr.r[2 * r + 1]; i += blockDim.x) p[i] = 0;
}
}  // namespace

int finish_blob(lc_column* col, const uint8_t* prefix_h, uint64_t prefix_len, cudaStream_t st) {
    int rc = stage_h2d(col->blob, prefix_h, prefix_len, st);
    if (rc) return rc;
    const Layout& F = col->lay;
    const uint64_t C = col->C, L = col->L;
    PadRanges pr;
    pr.n = 0;
    auto pad = [&](uint64_t off, uint64_t bytes) {
        const uint64_t end = off + bytes, padded = (end + 15) & ~(uint64_t)15;
        if (padded > end) {
            pr.r[2 * pr.n] = end;
            pr.r[2 * pr.n + 1] = padded;
            ++pr.n;
        }
    };
    pad(F.csb, 8 * (C + 1));
    pad(F.cwb, 8 * (C + 1));
    pad(F.icpt, (uint64_t)col->key_bytes * L);
    pad(F.slope, 8 * L);
    pad(F.bitoff, 4 * L);
    pad(F.start, 2 * L);
    pad(F.width, L);
    if (pr.n) {
        zero_pads<<<1, 256, 0, st>>>(col->blob, pr);
        note_launch();
        rc = cuda_status(cudaGetLastError());
        if (rc) return rc;
    }
    return cuda_status(cudaStreamSynchronize(st));
}

}  // namespace lcx
