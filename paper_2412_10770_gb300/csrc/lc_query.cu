// lc_query.cu -- decoding from K^c on the GPU: bulk and range decode, rank
// access and value lower_bound (Def. 1 decoding, Fig. 2 decoding stage
// K[i] = floor(f_j(i)) + Delta[i]; Table 2 / Sec. III-A segment search).
//
// Decode works on tiles of 2048 keys that never cross a chunk.  A CTA stages
// the model of every segment that meets its tile (intercept, slope, bit base,
// start, width) and the tile's payload words in shared memory, marks the
// segment starts in a 2048-bit map, and then every key finds its segment by a
// rank (popcount) on that map: no search per key.  Keys are written with
// consecutive threads on consecutive keys (coalesced).
#include <algorithm>
#include <mutex>
#include <vector>

#include "lc_internal.h"
#include "lc_math.cuh"

namespace lcx {
namespace {

constexpr int kDecThreads = 256;
constexpr uint32_t kMaxSegsPerTile = kTile + 1;
constexpr size_t kDecSmem = (size_t)kMaxSegsPerTile * 24 + 64 * 4 * 2 + (kTile + 4) * 4;

// Shared memory of one decode CTA when no tile meets more than ms segments.
__host__ __device__ constexpr size_t dec_smem(uint32_t ms) { return (size_t)ms * 24 + 64 * 4 * 2 + (kTile + 4) * 4; }

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

// Decode keys [lo_key, hi_key) of tile t into out[g - lo_key].
template <typename KT>
__device__ void decode_tile(const ColView& v, uint64_t t, uint64_t lo_key, uint64_t hi_key, KT* __restrict__ out,
                            uint8_t* smem, uint32_t smem_segs = 0) {
    const uint32_t ms = smem_segs ? smem_segs : v.max_tile_segs;
    uint64_t* s_icpt = (uint64_t*)smem;
    int64_t* s_slope = (int64_t*)(s_icpt + ms);
    uint64_t* s_meta = (uint64_t*)(s_slope + ms);
    uint32_t* s_bm = (uint32_t*)(s_meta + ms);
    uint32_t* s_pref = s_bm + 64;
    uint32_t* s_pay = s_pref + 64;
    __shared__ uint32_t s_win[2];

    const uint32_t tid = threadIdx.x;
    const TileDesc td = v.tiles[t];
    const uint64_t c = td.chunk;
    const uint64_t ckb = __ldg(v.ckb + c);
    const uint32_t local0 = (uint32_t)(td.key_begin - ckb);
    const uint32_t n = td.n;
    const uint64_t j0 = td.seg_lo;
    const uint32_t ns = (uint32_t)(td.seg_hi - j0 + 1);

    if (tid < 64) s_bm[tid] = 0;
    __syncthreads();
    for (uint32_t j = tid; j < ns; j += kDecThreads) {
        const uint64_t g = j0 + j;
        const uint32_t st = __ldg(v.start + g);
        const uint32_t w = __ldg(v.width + g);
        const uint32_t bo = __ldg(v.bitoff + g);
        s_icpt[j] = ld_icpt<KT>(v.icpt, g);
        s_slope[j] = __ldg(v.slope + g);
        // chunk-relative bit of the residual of key i (> st): bo + w (i - st - 1)
        const uint32_t base = bo - w * (st + 1);
        s_meta[j] = (uint64_t)base | ((uint64_t)st << 32) | ((uint64_t)w << 48);
        const uint32_t p = j ? st - local0 : 0;
        atomicOr(&s_bm[p >> 5], 1u << (p & 31u));
    }
    __syncthreads();
    if (tid < 32) {
        // exclusive popcount prefix over the 64 bitmap words, two per lane
        const uint32_t a = __popc(s_bm[2 * tid]), b = __popc(s_bm[2 * tid + 1]);
        uint32_t inc = a + b;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, off);
            if (tid >= (uint32_t)off) inc += o;
        }
        const uint32_t ex = inc - a - b;
        s_pref[2 * tid] = ex;
        s_pref[2 * tid + 1] = ex + a;
        if (tid == 0) {
            // payload window: from the tile's first residual to the end of its last
            const uint64_t m0 = s_meta[0], m1 = s_meta[ns - 1];
            const uint32_t st0 = (uint32_t)(m0 >> 32) & 0xFFFFu, w0 = (uint32_t)(m0 >> 48);
            const uint32_t st1 = (uint32_t)(m1 >> 32) & 0xFFFFu, w1 = (uint32_t)(m1 >> 48);
            const uint32_t lo_bit = (uint32_t)m0 + w0 * max(local0, st0 + 1);
            const uint32_t hi_bit = (uint32_t)m1 + w1 * (max(local0 + n - 1, st1) + 1);
            s_win[0] = lo_bit >> 5;
            s_win[1] = ((hi_bit + 31) >> 5) - (lo_bit >> 5) + 1;
        }
    }
    __syncthreads();
    const uint32_t wlo = s_win[0], cnt = s_win[1];
    const uint64_t pbase = 2 * __ldg(v.cwb + c) + wlo;
    const uint64_t plimit = 2 * v.W;
    for (uint32_t q = tid; q < cnt + 1; q += kDecThreads) {
        const uint64_t gi = pbase + q;
        s_pay[q] = gi < plimit ? __ldg(v.pay32 + gi) : 0u;
    }
    __syncthreads();

    const uint64_t kbeg = td.key_begin;
    uint32_t p0 = 0, p1 = n;
    if (lo_key > kbeg) p0 = (uint32_t)(lo_key - kbeg < (uint64_t)n ? lo_key - kbeg : (uint64_t)n);
    if (hi_key < kbeg + n) p1 = (uint32_t)(hi_key > kbeg ? hi_key - kbeg : 0);
    const uint32_t wbit = 32u * wlo;
    for (uint32_t p = p0 + tid; p < p1; p += kDecThreads) {
        const uint32_t wd = p >> 5;
        const uint32_t j = s_pref[wd] + __popc(s_bm[wd] & (0xFFFFFFFFu >> (31u - (p & 31u)))) - 1;
        const uint64_t meta = s_meta[j];
        const uint32_t st = (uint32_t)(meta >> 32) & 0xFFFFu, w = (uint32_t)(meta >> 48);
        const uint32_t i = local0 + p;
        uint64_t key = s_icpt[j];
        const uint32_t tt = i - st;
        if (tt) {
            const uint32_t lb = (uint32_t)meta + w * i - wbit;
            const uint32_t z = extract_bits(s_pay[lb >> 5], s_pay[(lb >> 5) + 1], lb & 31u, w);
            key += (uint64_t)(line_at(s_slope[j], tt) + (int64_t)unzigzag32(z));
        }
        out[kbeg + p - lo_key] = (KT)key;
    }
    __syncthreads();
}

// Persistent: each CTA decodes tiles t0 + blockIdx.x, t0 + blockIdx.x + gridDim.x, ...
template <typename KT>
__global__ void __launch_bounds__(kDecThreads) decode_kernel(ColView v, uint64_t t0, uint64_t nt, uint64_t begin,
                                                             uint64_t end, KT* __restrict__ out) {
    extern __shared__ __align__(16) uint8_t smem[];
    for (uint64_t t = blockIdx.x; t < nt; t += gridDim.x) decode_tile<KT>(v, t0 + t, begin, end, out, smem);
}

// Work items of a multi-range decode: range r covers tiles
// [first[r], first[r] + ntiles[r]).
__global__ void range_tiles_kernel(ColView v, const uint64_t* __restrict__ begin, const uint64_t* __restrict__ count,
                                   uint64_t m, uint64_t* __restrict__ first, uint32_t* __restrict__ ntiles) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m; r += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = begin[r], cnt = count[r];
        if (cnt == 0 || b > v.N || cnt > v.N - b) {
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
__global__ void __launch_bounds__(kDecThreads)
decode_ranges_kernel(ColView v, const uint64_t* __restrict__ begin, const uint64_t* __restrict__ count,
                     const uint64_t* __restrict__ out_off, uint64_t m, const uint64_t* __restrict__ first,
                     const uint64_t* __restrict__ work_off, KT* __restrict__ out) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint64_t total = work_off[m];
    for (uint64_t w = blockIdx.x; w < total; w += gridDim.x) {
        uint64_t lo = 0, hi = m - 1;  // last r with work_off[r] <= w
        while (lo < hi) {
            const uint64_t mid = (lo + hi + 1) >> 1;
            if (work_off[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        const uint64_t r = lo;
        const uint64_t b = begin[r];
        decode_tile<KT>(v, first[r] + (w - work_off[r]), b, b + count[r], out + out_off[r], smem);
    }
}

// Key t of the segment whose record is r (Fig. 2: floor(f_j(i)) + Delta[i]).
__device__ __forceinline__ uint64_t rec_key(const ColView& v, const SegRec& r, uint32_t t) {
    if (t == 0) return r.icpt;
    const uint32_t w = (uint32_t)(r.kstart_w >> 56);
    const int64_t line = line_at(r.slope, t);
    if (w == 0) return r.icpt + (uint64_t)line;
    const uint64_t pos = r.bit1 + (uint64_t)w * (t - 1);
    const uint64_t wi = pos >> 5;  // < 2W: the residual's bits lie inside the payload
    const uint32_t lo = __ldg(v.pay32 + wi);
    const uint32_t hi = wi + 1 < 2 * v.W ? __ldg(v.pay32 + wi + 1) : 0u;
    return r.icpt + (uint64_t)(line + (int64_t)unzigzag32(extract_bits(lo, hi, (uint32_t)(pos & 31u), w)));
}

__device__ __forceinline__ SegRec load_rec(const SegRec* p) {
    const ulonglong2* q = (const ulonglong2*)p;
    const ulonglong2 a = __ldg(q), b = __ldg(q + 1);
    SegRec r;
    r.icpt = a.x;
    r.slope = (int64_t)a.y;
    r.kstart_w = b.x;
    r.bit1 = b.y;
    return r;
}

constexpr uint64_t kKeyMask = (1ull << 56) - 1;

// Rank access: the segment of key i comes from one rank word (anchor bits +
// anchors before), its model from one 32-byte record, its residual from the
// payload: three dependent loads.  i < v.N.
__device__ __forceinline__ uint64_t access_one(const ColView& v, uint64_t i) {
    const ulonglong2 rw = __ldg((const ulonglong2*)(v.rank + (i >> 6)));
    const uint64_t j = rw.y + __popcll(rw.x & (~0ull >> (63u - (uint32_t)(i & 63u)))) - 1;
    const SegRec r = load_rec(v.recs + j);
    return rec_key(v, r, (uint32_t)(i - (r.kstart_w & kKeyMask)));
}

template <typename KT>
__global__ void access_kernel(ColView v, const uint64_t* __restrict__ idx, uint64_t m, KT* __restrict__ out) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < m; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = idx[q];
        if (i >= v.N) {
            atomicOr(v.status, kStOutOfRange);
            out[q] = 0;
            continue;
        }
        out[q] = (KT)access_one(v, i);
    }
}

// Entry k of the top intercept level: from `top_keys` when staged, else from
// the level itself.
template <typename KT>
__device__ __forceinline__ uint64_t top_at(const ColView& v, const uint64_t* top_keys, uint64_t k) {
    if (top_keys) return top_keys[k];
    return v.top ? __ldg(v.level[v.top] + k) : ld_icpt<KT>(v.icpt, k);
}

// Value lower_bound: the last segment whose intercept (its first key) is < x is
// found through the 16-ary sampled intercept levels (top level in shared
// memory, the next ones L2-resident, the last a 128-byte run of seg_icpt); then
// the segment's own line brackets the answer: every key lies within
// R = 2^(w-1) of floor(f), so keys before t < (dx - R)/s are < x and the key at
// t >= (dx + R + 1)/s is >= x (s = slope / 2^32, dx = x - intercept).  A
// binary search inside the bracket finishes.
template <typename KT>
__device__ uint64_t lower_bound_one(const ColView& v, uint64_t x, const uint64_t* top_keys) {
    const uint32_t top = v.top;
    const uint64_t ntop = top ? v.level_n[top] : v.L;
    if (v.L == 0 || top_at<KT>(v, top_keys, 0) >= x) return 0;
    uint64_t lo = 0, hi = ntop - 1;  // last entry < x
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        if (top_at<KT>(v, top_keys, mid) < x) lo = mid;
        else hi = mid - 1;
    }
    for (int d = (int)top - 1; d >= 0; --d) {
        const uint64_t nd = d ? v.level_n[d] : v.L;
        const uint64_t base = 16 * lo;
        uint64_t a = base, b = min(base + 16, nd) - 1;
        while (a < b) {
            const uint64_t mid = (a + b + 1) >> 1;
            const uint64_t key = d ? __ldg(v.level[d] + mid) : ld_icpt<KT>(v.icpt, mid);
            if (key < x) a = mid;
            else b = mid - 1;
        }
        lo = a;
    }
    const uint64_t j = lo;
    const SegRec r = load_rec(v.recs + j);
    const uint64_t ks = r.kstart_w & kKeyMask;
    const uint64_t ke = j + 1 < v.L ? (__ldg(&v.recs[j + 1].kstart_w) & kKeyMask) : v.N;
    const uint32_t n = (uint32_t)(ke - ks);
    uint32_t a = 1, b = n;  // first t in [1, n) with key(t) >= x, or n
    if (n >= 32 && r.slope > 0) {
        const uint32_t w = (uint32_t)(r.kstart_w >> 56);
        const float s = (float)r.slope * 2.3283064365386963e-10f;  // keys per index
        const float th = (float)(x - r.icpt) / s;
        const float dl = ((float)((1u << w) >> 1) + 1.0f) / s + 2.0f;
        const float fa = th - dl, fb = th + dl + 1.0f;
        a = fa <= 1.0f ? 1u : (fa >= (float)n ? n : (uint32_t)fa);
        b = fb <= 1.0f ? 1u : (fb >= (float)n ? n : (uint32_t)fb);
        if (a > b) a = b;
    }
    while (a < b) {
        const uint32_t mid = (a + b) >> 1;
        if (rec_key(v, r, mid) < x) a = mid + 1;
        else b = mid;
    }
    return ks + a;
}

template <typename KT>
__global__ void __launch_bounds__(256) lower_bound_kernel(ColView v, const KT* __restrict__ vals, uint64_t m,
                                                          uint64_t* __restrict__ out) {
    extern __shared__ uint64_t s_top[];
    const uint64_t ntop = v.top ? v.level_n[v.top] : v.L;
    for (uint64_t k = threadIdx.x; k < ntop; k += blockDim.x) s_top[k] = top_at<KT>(v, nullptr, k);
    __syncthreads();
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < m; q += (uint64_t)gridDim.x * blockDim.x)
        out[q] = lower_bound_one<KT>(v, (uint64_t)vals[q], s_top);
}

// ------------------------------------------------------------------ serving: multi-column batches

// Access and lower_bound requests of one batch, over any of the server's
// columns: query q belongs to the last request whose qoff <= q.
template <typename KT>
__global__ void serve_query_kernel(const ColView* __restrict__ views, const SrvReq* __restrict__ reqs, uint32_t nreq,
                                   uint64_t nq, const uint64_t* __restrict__ qin, uint64_t* __restrict__ qout,
                                   uint32_t* __restrict__ status) {
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
                qout[q] = access_one(v, x);
            }
        } else {
            qout[q] = lower_bound_one<KT>(v, x, nullptr);
        }
    }
}

// Range decodes of one batch: work item w is tile first_tile + (w - work_off[r])
// of request r, written to that request's own device buffer.
template <typename KT>
__global__ void __launch_bounds__(kDecThreads)
serve_decode_kernel(const ColView* __restrict__ views, const SrvReq* __restrict__ reqs, uint32_t nreq,
                    const uint64_t* __restrict__ work_off, uint32_t smem_segs) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint64_t total = work_off[nreq];
    for (uint64_t w = blockIdx.x; w < total; w += gridDim.x) {
        uint32_t lo = 0, hi = nreq - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (work_off[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        const SrvReq& rq = reqs[lo];
        decode_tile<KT>(views[rq.col], rq.first_tile + (w - work_off[lo]), rq.begin, rq.begin + rq.count,
                        (KT*)rq.out, smem, smem_segs);
    }
}

// Derived directories: segment records and rank bits (one CTA per chunk).
template <typename KT>
__global__ void rec_kernel(ColView v, SegRec* __restrict__ recs, RankWord* __restrict__ rank) {
    const uint64_t c = blockIdx.x;
    const uint64_t ckb = v.ckb[c], bit0 = 64 * v.cwb[c];
    for (uint64_t j = v.csb[c] + threadIdx.x; j < v.csb[c + 1]; j += blockDim.x) {
        const uint64_t k = ckb + v.start[j];
        SegRec r;
        r.icpt = ld_icpt<KT>(v.icpt, j);
        r.slope = v.slope[j];
        r.kstart_w = k | ((uint64_t)v.width[j] << 56);
        r.bit1 = bit0 + v.bitoff[j];
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

template <typename KT>
__global__ void level_kernel(ColView v, uint64_t* __restrict__ lvl, uint64_t n, uint64_t stride) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x)
        lvl[k] = ld_icpt<KT>(v.icpt, k * stride);
}

__global__ void tile_dir_kernel(ColView v, TileDesc* __restrict__ tiles, uint32_t* __restrict__ max_segs) {
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
    static bool done = false;
    if (done) return LC_OK;
    cudaError_t e = cudaFuncSetAttribute(decode_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDecSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(decode_ranges_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDecSmem);
    if (e != cudaSuccess) return cuda_status(e);
    done = true;
    return LC_OK;
}

}  // namespace

int build_derived(lc_column* col, cudaStream_t st) {
    const uint64_t C = col->C, L = col->L, N = col->N;
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
    int rc = cuda_status(cudaMemcpyAsync(col->chunk_tile_begin, ctb.data(), 8 * (C + 1), cudaMemcpyHostToDevice, st));
    if (rc) return rc;
    rc = cuda_status(cudaMemsetAsync(col->status, 0, 4, st));
    if (rc) return rc;

    // segment records, rank words, sampled intercept levels
    const uint64_t nw = (N + 63) / 64;
    uint32_t top = 0;
    uint64_t level_n[kMaxLevels] = {L};
    uint64_t level_off[kMaxLevels] = {0};
    uint64_t lv_total = 0;
    while (level_n[top] > kTopMax && top + 1 < (uint32_t)kMaxLevels) {
        ++top;
        level_n[top] = (level_n[top - 1] + 15) / 16;
        level_off[top] = lv_total;
        lv_total += level_n[top];
    }
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t off_rank = al(sizeof(SegRec) * L);
    const size_t off_lv = al(off_rank + sizeof(RankWord) * nw);
    const size_t bytes2 = al(off_lv + 8 * lv_total) + 256;
    if (cudaMallocAsync((void**)&col->derived2, bytes2, st) != cudaSuccess) {
        col->derived2 = nullptr;
        return LC_ERR_NOMEM;
    }
    SegRec* recs = (SegRec*)col->derived2;
    RankWord* rank = (RankWord*)(col->derived2 + off_rank);
    uint64_t* lv = (uint64_t*)(col->derived2 + off_lv);
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
    for (int d = 0; d < kMaxLevels; ++d) {
        v.level[d] = (d && d <= (int)top) ? lv + level_off[d] : nullptr;
        v.level_n[d] = d <= (int)top ? level_n[d] : 0;
    }
    v.top = top;
    v.key_bytes = col->key_bytes;
    v.status = col->status;
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
        tile_dir_kernel<<<(unsigned)((col->ntiles + 255) / 256), 256, 0, st>>>(v, col->tiles, col->status + 1);
        if (col->key_bytes == 4) rec_kernel<uint32_t><<<(unsigned)C, 128, 0, st>>>(v, recs, rank);
        else rec_kernel<uint64_t><<<(unsigned)C, 128, 0, st>>>(v, recs, rank);
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
        for (uint32_t d = 1; !rc && d <= top; ++d) {
            uint64_t stride = 1;
            for (uint32_t e = 0; e < d; ++e) stride *= 16;
            const unsigned gl = (unsigned)std::min<uint64_t>((level_n[d] + 255) / 256, 65535);
            if (col->key_bytes == 4) level_kernel<uint32_t><<<gl, 256, 0, st>>>(v, lv + level_off[d], level_n[d], stride);
            else level_kernel<uint64_t><<<gl, 256, 0, st>>>(v, lv + level_off[d], level_n[d], stride);
            note_launch();
            rc = cuda_status(cudaGetLastError());
        }
        cudaFreeAsync(t, st);
        if (rc) return rc;
        uint32_t ms = 0;
        rc = cuda_status(cudaMemcpyAsync(&ms, col->status + 1, 4, cudaMemcpyDeviceToHost, st));
        if (rc) return rc;
        rc = cuda_status(cudaStreamSynchronize(st));
        if (rc) return rc;
        v.max_tile_segs = std::max<uint32_t>(ms, 1);
        return LC_OK;
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

template <typename KT>
static int launch_decode(const lc_column* col, uint64_t t0, uint64_t nt, uint64_t begin, uint64_t count, void* out,
                         cudaStream_t st) {
    int rc = set_smem<KT>();
    if (rc) return rc;
    const size_t smem = dec_smem(col->view.max_tile_segs);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decode_kernel<KT>, kDecThreads, smem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    const uint64_t grid = std::min<uint64_t>(nt, (uint64_t)sm_count() * occ);
    {
        KTime kt("decode", st);
        decode_kernel<KT><<<(unsigned)grid, kDecThreads, smem, st>>>(col->view, t0, nt, begin, begin + count, (KT*)out);
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

int decode_ranges(const lc_column* col, const uint64_t* begin, const uint64_t* count, const uint64_t* out_off,
                  uint64_t m, void* out, cudaStream_t st) {
    if (m == 0) return LC_OK;
    const size_t tmp_b = scan_tmp_bytes(m);
    const size_t bytes = 8 * m + 4 * m + 8 * (m + 1) + tmp_b + 64;
    uint8_t* p = nullptr;
    if (cudaMallocAsync((void**)&p, bytes, st) != cudaSuccess) return LC_ERR_NOMEM;
    uint64_t* first = (uint64_t*)p;
    uint64_t* work_off = first + m;
    uint32_t* ntiles = (uint32_t*)(work_off + m + 1);
    void* tmp = (void*)(((uintptr_t)(ntiles + m) + 15) & ~(uintptr_t)15);
    range_tiles_kernel<<<(unsigned)std::min<uint64_t>((m + 255) / 256, 4096), 256, 0, st>>>(col->view, begin, count,
                                                                                              m, first, ntiles);
    note_launch();
    int rc = cuda_status(cudaGetLastError());
    if (!rc) rc = scan_exclusive(ntiles, work_off, m, ScanOp::Identity, tmp, tmp_b, st);
    if (!rc) {
        const unsigned grid = (unsigned)(sm_count() * 4);
        const size_t smem = dec_smem(col->view.max_tile_segs);
        if (col->key_bytes == 4) {
            if (!(rc = set_smem<uint32_t>())) {
                KTime kt("decode_ranges", st);
                decode_ranges_kernel<uint32_t><<<grid, kDecThreads, smem, st>>>(col->view, begin, count, out_off, m,
                                                                               first, work_off, (uint32_t*)out);
            }
        } else {
            if (!(rc = set_smem<uint64_t>())) {
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

int access(const lc_column* col, const uint64_t* idx, uint64_t m, void* out, cudaStream_t st) {
    if (m == 0) return LC_OK;
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
    const uint64_t ntop = v.top ? v.level_n[v.top] : v.L;
    const size_t smem = 8 * std::max<uint64_t>(ntop, 1);
    const unsigned grid = (unsigned)std::min<uint64_t>((m + 255) / 256, (uint64_t)sm_count() * 6);
    {
        KTime kt("lower_bound", st);
        if (col->key_bytes == 4)
            lower_bound_kernel<uint32_t><<<grid, 256, smem, st>>>(v, (const uint32_t*)vals, m, out);
        else
            lower_bound_kernel<uint64_t><<<grid, 256, smem, st>>>(v, (const uint64_t*)vals, m, out);
    }
    note_launch();
    return cuda_status(cudaGetLastError());
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
constexpr size_t kNoAllocScanBytes = 8 * ((kNoAllocMaxRanges + 4095) / 4096 + 1);    // scan partials
constexpr size_t kNoAllocScratchBytes = kNoAllocScanOff + kNoAllocScanBytes;

__device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
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
                          uint64_t m, void* out, cudaStream_t st) {
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
    range_tiles_kernel<<<(unsigned)std::min<uint64_t>((m + 255) / 256, 4096), 256, 0, st>>>(col->view, begin, count,
                                                                                              m, first, ntiles);
    note_launch();
    rc = cuda_status(cudaGetLastError());
    if (!rc) rc = scan_exclusive(ntiles, work_off, m, ScanOp::Identity, tmp, kNoAllocScanBytes, st);
    if (rc) return rc;
    const unsigned grid = (unsigned)(sm_count() * 4);
    if (col->key_bytes == 4) {
        if ((rc = set_smem<uint32_t>())) return rc;
        decode_ranges_kernel<uint32_t><<<grid, kDecThreads, dec_smem(col->view.max_tile_segs), st>>>(col->view, begin, count, out_off, m, first,
                                                                           work_off, (uint32_t*)out);
    } else {
        if ((rc = set_smem<uint64_t>())) return rc;
        decode_ranges_kernel<uint64_t><<<grid, kDecThreads, dec_smem(col->view.max_tile_segs), st>>>(col->view, begin, count, out_off, m, first,
                                                                           work_off, (uint64_t*)out);
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
        const unsigned grid = (unsigned)std::min<uint64_t>(nwork, (uint64_t)sm_count() * 4);
        if (key_bytes == 4) {
            static bool done = false;
            if (!done) {
                if ((rc = cuda_status(cudaFuncSetAttribute(serve_decode_kernel<uint32_t>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDecSmem))))
                    return rc;
                done = true;
            }
            serve_decode_kernel<uint32_t><<<grid, kDecThreads, smem, st>>>(views_d, dreqs_d, ndreq, work_off_d,
                                                                          max_tile_segs);
        } else {
            static bool done = false;
            if (!done) {
                if ((rc = cuda_status(cudaFuncSetAttribute(serve_decode_kernel<uint64_t>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDecSmem))))
                    return rc;
                done = true;
            }
            serve_decode_kernel<uint64_t><<<grid, kDecThreads, smem, st>>>(views_d, dreqs_d, ndreq, work_off_d,
                                                                          max_tile_segs);
        }
        note_launch();
        if ((rc = cuda_status(cudaGetLastError()))) return rc;
    }
    return LC_OK;
}

uint64_t tile_of_key(const lc_column* col, uint64_t i) { return host_tile_of(col, i); }

}  // namespace lcx
