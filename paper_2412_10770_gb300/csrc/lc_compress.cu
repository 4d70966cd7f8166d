// lc_compress.cu -- the compression path on the GPU: eps-PLA fit (Def. 2,
// Eq. (1)), residual widths and packing (Sec. II-A), all in exact integer
// arithmetic so that the bytes equal those of the CPU definition.
//
// Pipeline for C chunks (each chunk is independent: segments never cross one):
//   fit_kernel    one CTA per chunk.  The chunk is split into 64-key blocks.
//                 (S) every thread runs the greedy cone from its block's first
//                 key ("speculative" anchors), following the block's last
//                 segment past the block end; (F) assuming the true segment that
//                 enters block k ends where block k-1's speculation says, every
//                 thread re-walks its block until it meets a speculative anchor
//                 (from there on the speculation is exact: the greedy from a
//                 given anchor is deterministic); (R) one warp chains the blocks
//                 in order, using (S)/(F) whenever their assumption holds and
//                 walking the cone itself (32 keys per step) otherwise.  Output:
//                 one anchor bit per key and the segment count per chunk.
//   scan          chunk_seg_begin.
//   model_kernel  one CTA per chunk.  Every segment's cone is the intersection
//                 of its keys' slope intervals, so with the anchors known it is a
//                 segmented max/min over keys (exact rational comparisons, one
//                 division per segment edge).  Then the slope (floor midpoint),
//                 the width (bit length of the largest zigzag residual) and the
//                 bit offsets.  Writes the segment arrays of the blob.
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
constexpr uint32_t kInvalid = 0xFFFFFFFEu;  // (F) had no entry point
constexpr uint32_t kCap = 64;               // (S)/(F) follow a segment at most this far past the block
constexpr int kFitThreads = 256;
constexpr int kModelThreads = 256;
constexpr int kPackThreads = 256;
constexpr uint32_t kWin = 2048;             // keys per pack window
constexpr uint32_t kMaxBlocks = kMaxChunk / kBlock;
constexpr uint32_t kWalkAhead = 8 * 32;     // keys the warp walk prefetches ahead of its step

template <typename KT>
__device__ __forceinline__ uint64_t ldk(const KT* __restrict__ K, uint32_t i) {
    return (uint64_t)__ldg(K + i);
}

// Next anchor after anchor x: the first key that empties the cone, or `limit`
// if the segment reaches it (n when limit == n, kNone for an earlier limit).
template <typename KT>
__device__ uint32_t greedy_end(const KT* __restrict__ K, uint32_t x, uint32_t limit, uint32_t n,
                               int64_t eps, const uint64_t* __restrict__ magic) {
    uint64_t kx = ldk(K, x);
    int64_t LO = INT64_MIN, HI = INT64_MAX;
    for (uint32_t i = x + 1; i < limit; ++i) {
        uint64_t D = ldk(K, i) - kx;
        if (!cone_step(D, i - x, eps, LO, HI, magic)) return i;
    }
    return limit >= n ? n : kNone;
}

// The same greedy with a whole warp: each step tests 32 keys against the cone
// carried in from the previous step (two line evaluations per key); only keys
// that move an edge pay for a division, and an inclusive max/min scan over the
// lanes gives the cone after every key, hence the first key that empties it.
// Called with all 32 lanes active and warp-uniform arguments.
template <typename KT>
__device__ uint32_t warp_walk(const KT* __restrict__ K, uint32_t x, uint32_t n, int64_t eps,
                              uint32_t lane, const uint64_t* __restrict__ magic) {
    const uint64_t kx = ldk(K, x);
    int64_t LO = INT64_MIN, HI = INT64_MAX;
    uint32_t p = x + 1;
    while (p < n) {
        const uint32_t i = p + lane;
        const bool valid = i < n;
        const uint32_t d = i - x;
        // keep the keys of the steps ahead on their way into L2
        if (i + kWalkAhead < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(K + i + kWalkAhead));
        uint64_t D = valid ? ldk(K, i) - kx : 0;
        bool fits = false, tlo = false, thi = false;
        int64_t dlo = 0, dhi = 0;
        if (valid && D < (1ull << 48)) {
            dlo = (int64_t)D - eps;
            dhi = (int64_t)D + eps;
            const int64_t pl = line_at(LO, d), ph = line_at(HI, d);
            fits = pl <= dhi && ph >= dlo;
            tlo = fits && pl < dlo;
            thi = fits && ph > dhi;
        }
        const uint32_t failm = __ballot_sync(0xFFFFFFFFu, !fits);
        const uint32_t ff = failm ? (uint32_t)(__ffs(failm) - 1) : 32u;
        const uint32_t below = ff >= 32 ? 0xFFFFFFFFu : ((1u << ff) - 1u);
        const uint32_t need = __ballot_sync(0xFFFFFFFFu, tlo || thi) & below;
        if (need == 0) {
            if (ff < 32) return min(p + ff, n);
            p += 32;
            continue;
        }
        int64_t mylo = INT64_MIN, myhi = INT64_MAX;
        if (lane < ff) {
            if (tlo) mylo = ceil_q32(dlo, d, magic);
            if (thi) myhi = ceil_q32(dhi + 1, d, magic) - 1;
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t a = __shfl_up_sync(0xFFFFFFFFu, mylo, off);
            const int64_t b = __shfl_up_sync(0xFFFFFFFFu, myhi, off);
            if (lane >= (uint32_t)off) {
                mylo = max(mylo, a);
                myhi = min(myhi, b);
            }
        }
        const int64_t clo = max(LO, mylo), chi = min(HI, myhi);
        const uint32_t badm = __ballot_sync(0xFFFFFFFFu, lane >= ff || clo > chi);
        const uint32_t bk = badm ? (uint32_t)(__ffs(badm) - 1) : 32u;
        if (bk > 0) {
            LO = __shfl_sync(0xFFFFFFFFu, clo, bk - 1);
            HI = __shfl_sync(0xFFFFFFFFu, chi, bk - 1);
        }
        if (bk < 32) return min(p + bk, n);
        p += 32;
    }
    return n;
}

// ------------------------------------------------------------------ fit

template <typename KT>
__global__ void __launch_bounds__(kFitThreads)
fit_kernel(const KT* __restrict__ keys, const ChunkDesc* __restrict__ chunks, uint32_t* __restrict__ tbits,
           uint32_t* __restrict__ counts, uint32_t* __restrict__ status) {
    __shared__ uint64_t s_spec[kMaxBlocks];
    __shared__ uint64_t s_fix[kMaxBlocks];  // (F) anchors; overwritten in place by (R) with the true ones
    __shared__ uint32_t s_exitS[kMaxBlocks];
    __shared__ uint32_t s_exitF[kMaxBlocks];
    __shared__ uint8_t s_sync[kMaxBlocks];

    const ChunkDesc cd = chunks[blockIdx.x];
    const KT* __restrict__ K = keys + cd.key_begin;
    const uint32_t n = cd.n;
    const int64_t eps = cd.eps;
    const uint32_t nblk = (n + kBlock - 1) / kBlock;
    const uint64_t* __restrict__ magic = g_magic;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;

    // (S) speculative greedy from every block start; also the sortedness check.
    bool unsorted = false;
    for (uint32_t k = tid; k < nblk; k += kFitThreads) {
        const uint32_t b = k * kBlock, e = min(b + kBlock, n);
        if (b == 0 && cd.check_prev) unsorted |= __ldg(K - 1) > __ldg(K);
        for (uint32_t i = max(b, 1u); i < e; ++i) unsorted |= ldk(K, i - 1) > ldk(K, i);
        uint64_t mask = 0;
        uint32_t x = b, ex;
        for (;;) {
            mask |= 1ull << (x - b);
            const uint32_t y = greedy_end(K, x, min(n, e + kCap), n, eps, magic);
            if (y == kNone || y >= e) {
                ex = y;
                break;
            }
            x = y;
        }
        s_spec[k] = mask;
        s_exitS[k] = ex;
    }
    if (unsorted) atomicOr(status, kStUnsorted);
    __syncthreads();

    // (F) re-walk block k from the entry that block k-1's speculation predicts,
    // until a speculative anchor is met.
    for (uint32_t k = tid; k < nblk; k += kFitThreads) {
        if (k == 0) {
            s_fix[0] = 0;
            s_exitF[0] = kInvalid;
            s_sync[0] = 0xFF;
            continue;
        }
        uint32_t x = s_exitS[k - 1];
        if (x == kNone) {
            s_fix[k] = 0;
            s_exitF[k] = kInvalid;
            s_sync[k] = 0xFF;
            continue;
        }
        const uint32_t b = k * kBlock, e = min(b + kBlock, n);
        const uint64_t sm = s_spec[k];
        uint64_t fm = 0;
        uint32_t sync = 0xFF;
        while (x < e) {
            if ((sm >> (x - b)) & 1ull) {
                sync = x - b;
                break;
            }
            fm |= 1ull << (x - b);
            x = greedy_end(K, x, min(n, e + kCap), n, eps, magic);
            if (x == kNone) break;
        }
        s_fix[k] = fm;
        s_sync[k] = (uint8_t)sync;
        s_exitF[k] = sync != 0xFF ? s_exitS[k] : x;
    }
    __syncthreads();

    // (R) chain the blocks in order: the true anchors.
    if (warp == 0) {
        uint32_t x = 0, total = 0;
        for (uint32_t k = 0; k < nblk; ++k) {
            const uint32_t b = k * kBlock, e = min(b + kBlock, n);
            uint64_t mask = 0;
            if (x < e) {
                uint32_t xn;
                if (k == 0) {
                    mask = s_spec[0];
                    xn = s_exitS[0];
                } else if (x == s_exitS[k - 1] && s_exitF[k] != kInvalid) {
                    mask = s_fix[k];
                    const uint32_t so = s_sync[k];
                    if (so != 0xFF) mask |= s_spec[k] & (~0ull << so);
                    xn = s_exitF[k];
                } else {
                    const uint64_t sm = s_spec[k];
                    xn = x;
                    while (xn < e) {
                        if ((sm >> (xn - b)) & 1ull) {
                            mask |= sm & (~0ull << (xn - b));
                            xn = s_exitS[k];
                            break;
                        }
                        mask |= 1ull << (xn - b);
                        xn = warp_walk(K, xn, n, eps, lane, magic);
                    }
                }
                if (xn == kNone) {
                    const uint32_t la = b + 63u - (uint32_t)__clzll((long long)mask);
                    xn = warp_walk(K, la, n, eps, lane, magic);
                }
                x = xn;
            }
            __syncwarp();
            if (lane == 0) s_fix[k] = mask;
            total += __popcll(mask);
        }
        if (lane == 0) counts[blockIdx.x] = total;
    }
    __syncthreads();

    // anchor bitmap of the chunk, 32 bits per word
    uint32_t* __restrict__ T = tbits + cd.bitword_begin;
    const uint32_t nwords = (n + 31) / 32;
    for (uint32_t wd = tid; wd < nwords; wd += kFitThreads)
        T[wd] = (uint32_t)(s_fix[wd >> 1] >> (32 * (wd & 1u)));
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

// Rational running extremes of one piece of a segment: max over keys of
// (D - eps)/d and min over keys of (D + eps + 1)/d.
struct Cone {
    int64_t X;   // numerator of the max lower slope / 2^32
    uint64_t Y;  // numerator of the min upper slope / 2^32
    uint32_t E, F;
    uint32_t has;
};

__device__ __forceinline__ void cone_add(Cone& c, int64_t xl, uint64_t yh, uint32_t d) {
    if (!c.has) {
        c.X = xl; c.E = d; c.Y = yh; c.F = d; c.has = 1;
        return;
    }
    if (xl * (int64_t)c.E > c.X * (int64_t)d) { c.X = xl; c.E = d; }
    if (yh * (uint64_t)c.F < c.Y * (uint64_t)d) { c.Y = yh; c.F = d; }
}

__device__ __forceinline__ void cone_merge(Cone& c, const Cone& o) {
    if (!o.has) return;
    if (!c.has) { c = o; return; }
    if (o.X * (int64_t)c.E > c.X * (int64_t)o.E) { c.X = o.X; c.E = o.E; }
    if (o.Y * (uint64_t)c.F < c.Y * (uint64_t)o.F) { c.Y = o.Y; c.F = o.F; }
}

// Slope of a closed segment: the floor midpoint of [LO, HI] with
// LO = ceil(2^32 X/E) and HI = min(ceil(2^32 Y/F) - 1, INT64_MAX); 0 for a
// single key.
__device__ __forceinline__ int64_t cone_slope(const Cone& c, const uint64_t* __restrict__ magic) {
    if (!c.has) return 0;
    const int64_t LO = ceil_q32(c.X, c.E, magic);
    int64_t HI;
    if (c.Y >= ((uint64_t)c.F << 31)) HI = INT64_MAX;
    else HI = ceil_q32((int64_t)c.Y, c.F, magic) - 1;
    return LO + (int64_t)(((uint64_t)HI - (uint64_t)LO) >> 1);
}

__device__ __forceinline__ bool tbit(const uint32_t* s_T, uint32_t i) { return (s_T[i >> 5] >> (i & 31u)) & 1u; }

// First anchor strictly after position a (n if none), scanning words.
__device__ __forceinline__ uint32_t next_anchor(const uint32_t* s_T, uint32_t a, uint32_t n) {
    uint32_t i = a + 1;
    if (i >= n) return n;
    uint32_t wd = i >> 5;
    uint32_t bits = s_T[wd] & (0xFFFFFFFFu << (i & 31u));
    const uint32_t nw = (n + 31) >> 5;
    while (!bits) {
        if (++wd >= nw) return n;
        bits = s_T[wd];
    }
    return min(n, wd * 32u + (uint32_t)(__ffs(bits) - 1));
}

template <typename KT>
__global__ void __launch_bounds__(kModelThreads)
model_kernel(const KT* __restrict__ keys, const ChunkDesc* __restrict__ chunks,
             const uint32_t* __restrict__ tbits, const uint64_t* __restrict__ csb, KT* __restrict__ icpt,
             int64_t* __restrict__ slope, uint32_t* __restrict__ bitoff, uint16_t* __restrict__ start,
             uint8_t* __restrict__ width, uint32_t* __restrict__ chunk_bits) {
    __shared__ uint32_t s_T[kMaxChunk / 32];
    __shared__ Cone s_part[kModelThreads];
    __shared__ Cone s_head[kModelThreads];
    __shared__ uint32_t s_head_anchor[kModelThreads], s_head_end[kModelThreads], s_cnt[kModelThreads];
    __shared__ uint64_t s_head_rank[kModelThreads];
    __shared__ int64_t s_head_M[kModelThreads];
    __shared__ uint32_t s_part_z[kModelThreads], s_head_z[kModelThreads];
    __shared__ uint32_t s_warp_u32[32];
    __shared__ int32_t s_warp_i32[32];

    const ChunkDesc cd = chunks[blockIdx.x];
    const KT* __restrict__ K = keys + cd.key_begin;
    const uint32_t n = cd.n;
    const int64_t eps = cd.eps;
    const uint64_t* __restrict__ magic = g_magic;
    const uint32_t tid = threadIdx.x;
    const uint32_t nwords = (n + 31) / 32;
    for (uint32_t wd = tid; wd < nwords; wd += kModelThreads) s_T[wd] = tbits[cd.bitword_begin + wd];
    __syncthreads();
    const uint64_t seg0 = csb[blockIdx.x];

    // runs of R keys (a multiple of 32) per thread
    const uint32_t per = (n + kModelThreads - 1) / kModelThreads;
    const uint32_t R = ((per + 31) / 32) * 32;
    const uint32_t r0 = min(n, tid * R), r1 = min(n, r0 + R);
    uint32_t cnt = 0;
    int32_t last = -1;
    for (uint32_t wd = r0 >> 5; wd < (r1 + 31) >> 5; ++wd) {
        const uint32_t bits = s_T[wd];
        cnt += __popc(bits);
        if (bits) last = (int32_t)(wd * 32 + 31 - __clz(bits));
    }
    s_cnt[tid] = cnt;
    uint32_t rank_total;
    const uint32_t rank_base = block_excl_scan<uint32_t>(cnt, AddOp(), 0u, s_warp_u32, &rank_total);
    const int32_t prev_anchor = block_excl_scan<int32_t>(last, MaxOp(), -1, s_warp_i32, nullptr);

    const bool run_empty = r0 >= r1;
    const bool starts_with_anchor = !run_empty && tbit(s_T, r0);
    const uint32_t a0 = starts_with_anchor ? r0 : (uint32_t)max(prev_anchor, 0);
    const uint64_t j0 = seg0 + (starts_with_anchor ? rank_base : rank_base - 1);

    // pass 1: cones
    Cone c{0, 0, 0, 0, 0};
    uint32_t cur_a = a0;
    uint64_t cur_j = j0;
    uint64_t ka = run_empty ? 0 : ldk(K, a0);
    bool first_piece = !starts_with_anchor;
    s_part[tid].has = 0;
    s_head[tid].has = 0;
    s_head_anchor[tid] = kNone;
    for (uint32_t i = r0; i < r1; ++i) {
        if (tbit(s_T, i)) {
            if (i != r0) {  // close the piece that ends here: complete unless it began before the run
                if (first_piece) {
                    s_part[tid] = c;
                } else {
                    slope[cur_j] = cone_slope(c, magic);
                    start[cur_j] = (uint16_t)cur_a;
                    icpt[cur_j] = (KT)ka;
                }
                ++cur_j;
            }
            cur_a = i;
            ka = ldk(K, i);
            c.has = 0;
            first_piece = false;
            continue;
        }
        const uint64_t D = ldk(K, i) - ka;
        cone_add(c, (int64_t)D - eps, D + (uint64_t)eps + 1, i - cur_a);
    }
    if (!run_empty) {
        if (first_piece) {
            s_part[tid] = c;
        } else if (r1 == n || tbit(s_T, r1)) {
            slope[cur_j] = cone_slope(c, magic);
            start[cur_j] = (uint16_t)cur_a;
            icpt[cur_j] = (KT)ka;
        } else {
            s_head[tid] = c;
            s_head_anchor[tid] = cur_a;
            s_head_rank[tid] = cur_j;
        }
    }
    __syncthreads();

    // heads: fold the pieces of the following runs that the segment spans
    const uint32_t nruns = (n + R - 1) / R;
    if (s_head_anchor[tid] != kNone) {
        Cone h = s_head[tid];
        uint32_t u = tid + 1;
        for (; u < nruns; ++u) {
            cone_merge(h, s_part[u]);
            if (s_cnt[u] > 0) break;
        }
        const uint32_t a = s_head_anchor[tid];
        const uint32_t end = u < nruns ? next_anchor(s_T, u * R - 1, n) : n;
        s_head_end[tid] = end;
        const int64_t M = cone_slope(h, magic);
        s_head_M[tid] = M;
        const uint64_t j = s_head_rank[tid];
        slope[j] = M;
        start[j] = (uint16_t)a;
        icpt[j] = (KT)ldk(K, a);
    }
    __syncthreads();

    // pass 2: residual widths
    uint32_t owned_bits = 0;
    {
        cur_a = a0;
        cur_j = j0;
        ka = run_empty ? 0 : ldk(K, a0);
        int64_t M = 0;
        if (!run_empty) M = starts_with_anchor ? slope[j0] : s_head_M[a0 / R];
        first_piece = !starts_with_anchor;
        uint32_t zmax = 0;
        s_part_z[tid] = 0;
        s_head_z[tid] = 0;
        for (uint32_t i = r0; i < r1; ++i) {
            if (tbit(s_T, i)) {
                if (i != r0) {
                    if (first_piece) {
                        s_part_z[tid] = zmax;
                    } else {
                        const uint32_t w = 32u - __clz(zmax);
                        width[cur_j] = (uint8_t)w;
                        owned_bits += w * (i - cur_a - 1);
                    }
                    ++cur_j;
                }
                cur_a = i;
                ka = ldk(K, i);
                first_piece = false;
                zmax = 0;
                // the slope of the segment starting here: its own (complete) or this run's head
                M = (s_head_anchor[tid] == i) ? s_head_M[tid] : slope[cur_j];
                continue;
            }
            const uint64_t D = ldk(K, i) - ka;
            const int64_t r = (int64_t)D - line_at(M, i - cur_a);
            zmax = max(zmax, zigzag32(r));
        }
        if (!run_empty && first_piece) s_part_z[tid] = zmax;
        if (!run_empty && !first_piece) {
            if (r1 == n || tbit(s_T, r1)) {
                const uint32_t w = 32u - __clz(zmax);
                width[cur_j] = (uint8_t)w;
                owned_bits += w * (r1 - cur_a - 1);
            } else {
                s_head_z[tid] = zmax;
            }
        }
    }
    __syncthreads();
    if (s_head_anchor[tid] != kNone) {
        uint32_t zmax = s_head_z[tid];
        for (uint32_t u = tid + 1; u < nruns; ++u) {
            zmax = max(zmax, s_part_z[u]);
            if (s_cnt[u] > 0) break;
        }
        const uint32_t w = 32u - __clz(zmax);
        width[s_head_rank[tid]] = (uint8_t)w;
        owned_bits += w * (s_head_end[tid] - s_head_anchor[tid] - 1);
    }

    // bit offsets: exclusive scan of the bits of the segments each run owns
    uint32_t total_bits;
    uint32_t bit = block_excl_scan<uint32_t>(owned_bits, AddOp(), 0u, s_warp_u32, &total_bits);
    if (!run_empty) {
        uint64_t j = starts_with_anchor ? j0 : j0 + 1;
        for (uint32_t wd = r0 >> 5; wd < (r1 + 31) >> 5; ++wd) {
            uint32_t bits = s_T[wd];
            while (bits) {
                const uint32_t a = wd * 32 + (uint32_t)(__ffs(bits) - 1);
                bits &= bits - 1;
                if (a < r0 || a >= r1) continue;
                const uint32_t end = (s_head_anchor[tid] == a) ? s_head_end[tid] : next_anchor(s_T, a, n);
                bitoff[j] = bit;
                bit += (uint32_t)width[j] * (end - a - 1);
                ++j;
            }
        }
    }
    if (tid == 0) chunk_bits[blockIdx.x] = total_bits;
}

// ------------------------------------------------------------------ pack

template <typename KT>
__global__ void __launch_bounds__(kPackThreads)
pack_kernel(const KT* __restrict__ keys, const ChunkDesc* __restrict__ chunks, const uint32_t* __restrict__ tbits,
            const uint64_t* __restrict__ csb, const uint64_t* __restrict__ cwb, const KT* __restrict__ icpt,
            const int64_t* __restrict__ slope, const uint32_t* __restrict__ bitoff,
            const uint16_t* __restrict__ start, const uint8_t* __restrict__ width, uint32_t* __restrict__ pay32) {
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

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;

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
    scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, op, part);
    scan_parts<<<1, kScanThreads, 0, st>>>(part, nb);
    scan_final<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, op, part, out);
    note_launch(3);
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ host pipeline

static int ensure_magic(int dev) {
    static bool done[64] = {false};
    if (dev < 0 || dev >= 64) return LC_ERR_INTERNAL;
    if (done[dev]) return LC_OK;
    std::vector<uint64_t> m(kMaxChunk, 0);
    for (uint32_t d = 2; d < kMaxChunk; ++d) {
        const unsigned __int128 two64 = (unsigned __int128)1 << 64;
        m[d] = (uint64_t)((two64 + d - 1) / d);
    }
    cudaError_t e = cudaMemcpyToSymbol(g_magic, m.data(), m.size() * sizeof(uint64_t));
    if (e != cudaSuccess) return cuda_status(e);
    done[dev] = true;
    return LC_OK;
}

template <typename KT>
static int run_pipeline(const KT* keys, const ChunkDesc* chunks_d, uint64_t C, uint32_t* tbits, uint32_t* counts,
                        uint64_t* csb, uint32_t* status, void* tmp, size_t tmp_bytes, lc_column* col,
                        cudaStream_t st, int stage) {
    uint8_t* blob = col->blob;
    const Layout& lay = col->lay;
    if (stage == 0) {
        fit_kernel<KT><<<(unsigned)C, kFitThreads, 0, st>>>(keys, chunks_d, tbits, counts, status);
        note_launch();
        int rc = cuda_status(cudaGetLastError());
        if (rc) return rc;
        return scan_exclusive(counts, csb, C, ScanOp::Identity, tmp, tmp_bytes, st);
    }
    model_kernel<KT><<<(unsigned)C, kModelThreads, 0, st>>>(
        keys, chunks_d, tbits, (const uint64_t*)(blob + lay.csb), (KT*)(blob + lay.icpt), (int64_t*)(blob + lay.slope),
        (uint32_t*)(blob + lay.bitoff), (uint16_t*)(blob + lay.start), (uint8_t*)(blob + lay.width), counts);
    note_launch();
    int rc = cuda_status(cudaGetLastError());
    if (rc) return rc;
    rc = scan_exclusive(counts, (uint64_t*)(blob + lay.cwb), C, ScanOp::BitsToEvenWords, tmp, tmp_bytes, st);
    if (rc) return rc;
    pack_kernel<KT><<<(unsigned)C, kPackThreads, 0, st>>>(
        keys, chunks_d, tbits, (const uint64_t*)(blob + lay.csb), (const uint64_t*)(blob + lay.cwb),
        (const KT*)(blob + lay.icpt), (const int64_t*)(blob + lay.slope), (const uint32_t*)(blob + lay.bitoff),
        (const uint16_t*)(blob + lay.start), (const uint8_t*)(blob + lay.width), (uint32_t*)(blob + lay.payload));
    note_launch();
    return cuda_status(cudaGetLastError());
}

int compress_impl(const void* keys_dev, int kb, const ChunkDesc* chunks_h, uint64_t C, uint64_t bitwords,
                  uint64_t payload_bound_words, cudaStream_t st, lc_column* col) {
    int rc = ensure_magic(col->device);
    if (rc) return rc;
    // scratch: chunk table, anchor bitmap, per-chunk counts, scan partials, status, csb
    const size_t tmp_bytes = scan_tmp_bytes(C);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t off_chunks = 0;
    const size_t off_bits = al(off_chunks + C * sizeof(ChunkDesc));
    const size_t off_counts = al(off_bits + bitwords * 4);
    const size_t off_tmp = al(off_counts + (C + 1) * 4);
    const size_t off_status = al(off_tmp + tmp_bytes);
    const size_t off_csb = al(off_status + 256);
    const size_t scratch_bytes = off_csb + (C + 1) * sizeof(uint64_t);
    uint8_t* scratch = nullptr;
    if (cudaMallocAsync((void**)&scratch, scratch_bytes, st) != cudaSuccess) return LC_ERR_NOMEM;
    ChunkDesc* chunks_d = (ChunkDesc*)(scratch + off_chunks);
    uint32_t* tbits = (uint32_t*)(scratch + off_bits);
    uint32_t* counts = (uint32_t*)(scratch + off_counts);
    void* tmp = scratch + off_tmp;
    uint32_t* status = (uint32_t*)(scratch + off_status);
    uint64_t* csb_tmp = (uint64_t*)(scratch + off_csb);
    uint64_t total = 0;
    uint32_t h_status = 0;
    auto fail = [&](int code) {
        cudaStreamSynchronize(st);
        cudaFreeAsync(scratch, st);
        return code;
    };

    rc = cuda_status(cudaMemcpyAsync(chunks_d, chunks_h, C * sizeof(ChunkDesc), cudaMemcpyHostToDevice, st));
    if (rc) return fail(rc);
    rc = cuda_status(cudaMemsetAsync(status, 0, 4, st));
    if (rc) return fail(rc);

    // stage 0: anchors and segment counts
    if (kb == 4)
        rc = run_pipeline<uint32_t>((const uint32_t*)keys_dev, chunks_d, C, tbits, counts, csb_tmp, status, tmp,
                                    tmp_bytes, col, st, 0);
    else
        rc = run_pipeline<uint64_t>((const uint64_t*)keys_dev, chunks_d, C, tbits, counts, csb_tmp, status, tmp,
                                    tmp_bytes, col, st, 0);
    if (rc) return fail(rc);
    rc = cuda_status(cudaMemcpyAsync(&total, csb_tmp + C, 8, cudaMemcpyDeviceToHost, st));
    if (rc) return fail(rc);
    rc = cuda_status(cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, st));
    if (rc) return fail(rc);
    rc = cuda_status(cudaStreamSynchronize(st));
    if (rc) return fail(rc);
    if (h_status & kStUnsorted) return fail(LC_ERR_UNSORTED);
    const uint64_t L = total;

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

    // stage 1: model, widths, payload
    if (kb == 4)
        rc = run_pipeline<uint32_t>((const uint32_t*)keys_dev, chunks_d, C, tbits, counts, csb_tmp, status, tmp,
                                    tmp_bytes, col, st, 1);
    else
        rc = run_pipeline<uint64_t>((const uint64_t*)keys_dev, chunks_d, C, tbits, counts, csb_tmp, status, tmp,
                                    tmp_bytes, col, st, 1);
    if (rc) return fail(rc);
    rc = cuda_status(cudaMemcpyAsync(&total, col->blob + lay.cwb + 8 * C, 8, cudaMemcpyDeviceToHost, st));
    if (rc) return fail(rc);
    rc = cuda_status(cudaStreamSynchronize(st));
    if (rc) return fail(rc);
    if (total > payload_bound_words) return fail(LC_ERR_INTERNAL);
    col->W = total;
    col->lay = make_layout(kb, C, L, col->W, col->NL, col->list_mode != 0);
    cudaFreeAsync(scratch, st);
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
    int rc = cuda_status(cudaMemcpyAsync(col->blob, prefix_h, prefix_len, cudaMemcpyHostToDevice, st));
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
