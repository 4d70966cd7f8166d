// lc_for.cu -- the frame-of-reference delta bit-packing baseline (block of 128
// keys) that the scale sweep compares the learned compressor against.  It is a
// conventional codec, not part of the paper's method: the paper compares its
// learned compressor with such codecs (Sec. II-C, Fig. 3a).
//
// Format "FOR1" (little-endian, every array 16-byte aligned, padding zero):
//   header, 32 bytes: magic "FOR1", key_bytes u32, N u64, B u64 (blocks of
//   128 keys, the last one ragged), W u64 (32-bit payload words);
//   block_base: the first key of every block (key_bytes each);
//   block_width: u8 per block, the bit length of the block's largest delta;
//   payload: u32 words.  Block b holds its 128 deltas d_0 = 0,
//   d_i = K[128b + i] - K[128b + i - 1] (0 past the last key) at w_b bits
//   each, delta i at bit i * w_b of the block's 4 w_b words; block b starts at
//   word 4 * (w_0 + ... + w_{b-1}).
//
// One warp handles one block: lane l owns deltas 4l .. 4l+3, so that its bits
// are one contiguous run and its four keys one 16- or 32-byte store.  Decode
// is an exclusive warp scan of the lanes' delta sums.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lc_internal.h"

struct lc_for {
    int device;
    uint32_t key_bytes;
    uint64_t N, B, W;
    uint64_t off_base, off_width, off_payload, total;
    uint8_t* blob;    // device, exact FOR1 bytes
    uint64_t* woff;   // device, derived: payload word offset of every block [B + 1]
    uint32_t* status; // device status word
};

namespace lcx {
namespace {

constexpr uint32_t kForBlock = 128;
constexpr int kForWarps = 8;  // blocks per CTA
constexpr int kForThreads = 32 * kForWarps;

__host__ __device__ inline uint64_t for_pad16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

// The lane's four keys of block b (keys past n repeat the last key, so that
// their deltas are 0) and the key before its first one.
template <typename KT>
__device__ __forceinline__ void for_lane_keys(const KT* __restrict__ K, uint64_t n, uint64_t b, uint32_t lane,
                                              uint64_t k[4], uint64_t* prev) {
    const uint64_t i0 = b * kForBlock + 4 * lane;
#pragma unroll
    for (uint32_t u = 0; u < 4; ++u) {
        const uint64_t i = i0 + u;
        k[u] = (uint64_t)__ldg(K + (i < n ? i : n - 1));
    }
    const uint64_t up = __shfl_up_sync(0xFFFFFFFFu, k[3], 1);
    *prev = lane ? up : k[0];  // delta 0 of the block is 0
}

__device__ __forceinline__ uint32_t bitlen64(uint64_t x) { return 64u - (uint32_t)__clzll((long long)x); }

// Widths and bases: one warp per block.  Also checks that the keys are
// non-decreasing (within the block and across the boundary with the previous
// block).
template <typename KT>
__global__ void __launch_bounds__(kForThreads)
for_width_kernel(const KT* __restrict__ K, uint64_t n, uint64_t B, KT* __restrict__ base, uint8_t* __restrict__ width,
                 uint32_t* __restrict__ words, uint32_t* __restrict__ status) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t b = (uint64_t)blockIdx.x * kForWarps + (threadIdx.x >> 5);
    if (b >= B) return;
    uint64_t k[4], prev;
    for_lane_keys(K, n, b, lane, k, &prev);
    uint32_t wmax = 0;
    bool bad = k[0] < prev;
    wmax = max(wmax, bitlen64(k[0] - prev));
#pragma unroll
    for (uint32_t u = 1; u < 4; ++u) {
        bad |= k[u] < k[u - 1];
        wmax = max(wmax, bitlen64(k[u] - k[u - 1]));
    }
    if (lane == 0 && b > 0) bad |= (uint64_t)__ldg(K + b * kForBlock - 1) > k[0];
    wmax = __reduce_max_sync(0xFFFFFFFFu, wmax);
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(status, kStUnsorted);
    if (lane == 0) {
        base[b] = (KT)k[0];
        width[b] = (uint8_t)wmax;
        words[b] = 4 * wmax;
    }
}

// Pack: lane l writes its four deltas as one contiguous run of 4w bits at bit
// 4lw of the block, OR-ed into the block's words in shared memory (at most 256
// words), which are then stored whole.
template <typename KT>
__global__ void __launch_bounds__(kForThreads)
for_pack_kernel(const KT* __restrict__ K, uint64_t n, uint64_t B, const uint8_t* __restrict__ width,
                const uint64_t* __restrict__ woff, uint32_t* __restrict__ payload) {
    __shared__ uint32_t s_buf[kForWarps][4 * 64 + 1];
    const uint32_t lane = threadIdx.x & 31u, wp = threadIdx.x >> 5;
    const uint64_t b = (uint64_t)blockIdx.x * kForWarps + wp;
    if (b >= B) return;
    uint32_t* buf = s_buf[wp];
    const uint32_t w = width[b];
    for (uint32_t q = lane; q < 4 * w + 1; q += 32) buf[q] = 0;
    __syncwarp();
    uint64_t k[4], prev;
    for_lane_keys(K, n, b, lane, k, &prev);
    if (w) {
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
            const uint64_t d = k[u] - (u ? k[u - 1] : prev);
            const uint32_t pos = (4 * lane + u) * w;
            const uint32_t q = pos >> 5, sh = pos & 31u;
            // the delta spans at most three words: bits [pos, pos + w) with w <= 64
            atomicOr(buf + q, (uint32_t)(d << sh));
            if (sh + w > 32) atomicOr(buf + q + 1, (uint32_t)(d >> (32 - sh)));
            if (sh + w > 64) atomicOr(buf + q + 2, (uint32_t)(d >> (64 - sh)));
        }
    }
    __syncwarp();
    uint32_t* __restrict__ dst = payload + woff[b];
    for (uint32_t q = lane; q < 4 * w; q += 32) dst[q] = buf[q];
}

// Decode: lane l extracts its four deltas from the block's words, sums them,
// and an exclusive warp scan of the sums gives the key before its first one.
template <typename KT>
__global__ void __launch_bounds__(kForThreads)
for_decode_kernel(const uint8_t* __restrict__ blob, uint64_t off_base, uint64_t off_width, uint64_t off_payload,
                  uint64_t n, uint64_t B, const uint64_t* __restrict__ woff, KT* __restrict__ out) {
    __shared__ uint32_t s_buf[kForWarps][4 * 64 + 2];
    const uint32_t lane = threadIdx.x & 31u, wp = threadIdx.x >> 5;
    const uint64_t b = (uint64_t)blockIdx.x * kForWarps + wp;
    if (b >= B) return;
    const KT* __restrict__ base = (const KT*)(blob + off_base);
    const uint32_t w = blob[off_width + b];
    const uint32_t* __restrict__ src = (const uint32_t*)(blob + off_payload) + woff[b];
    uint32_t* buf = s_buf[wp];
    for (uint32_t q = lane; q < 4 * w + 2; q += 32) buf[q] = q < 4 * w ? __ldg(src + q) : 0u;
    __syncwarp();
    uint64_t d[4];
    const uint64_t mask = w == 64 ? ~0ull : (1ull << w) - 1;
#pragma unroll
    for (uint32_t u = 0; u < 4; ++u) {
        const uint32_t pos = (4 * lane + u) * w;
        const uint32_t q = pos >> 5, sh = pos & 31u;
        const uint64_t lo = ((uint64_t)buf[q + 1] << 32) | buf[q];
        uint64_t v = lo >> sh;
        if (sh) v |= (uint64_t)buf[q + 2] << (64 - sh);
        d[u] = w ? v & mask : 0;
    }
    uint64_t s = d[0] + d[1] + d[2] + d[3];
    // inclusive warp scan of the lane sums
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t o = __shfl_up_sync(0xFFFFFFFFu, s, off);
        if (lane >= (uint32_t)off) s += o;
    }
    uint64_t key = (uint64_t)base[b] + s - (d[0] + d[1] + d[2] + d[3]);
    const uint64_t i0 = b * kForBlock + 4 * lane;
    KT v[4];
#pragma unroll
    for (uint32_t u = 0; u < 4; ++u) {
        key += d[u];
        v[u] = (KT)key;
    }
    if (i0 + 4 <= n) {
        if (sizeof(KT) == 8) {
            ulonglong2* o = (ulonglong2*)(out + i0);
            o[0] = make_ulonglong2((uint64_t)v[0], (uint64_t)v[1]);
            o[1] = make_ulonglong2((uint64_t)v[2], (uint64_t)v[3]);
        } else {
            *(uint4*)(out + i0) = make_uint4((uint32_t)v[0], (uint32_t)v[1], (uint32_t)v[2], (uint32_t)v[3]);
        }
    } else {
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u)
            if (i0 + u < n) out[i0 + u] = v[u];
    }
}

__global__ void for_zero_kernel(uint8_t* __restrict__ p, uint64_t a0, uint64_t a1, uint64_t c0, uint64_t c1) {
    for (uint64_t i = a0 + threadIdx.x; i < a1; i += blockDim.x) p[i] = 0;
    for (uint64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) p[i] = 0;
}

void for_layout(lc_for* f) {
    f->off_base = 32;
    f->off_width = f->off_base + for_pad16((uint64_t)f->key_bytes * f->B);
    f->off_payload = f->off_width + for_pad16(f->B);
    f->total = f->off_payload + 4 * f->W;
}

void for_free(lc_for* f) {
    if (!f) return;
    if (f->blob) cudaFree(f->blob);
    if (f->woff) cudaFree(f->woff);
    if (f->status) cudaFree(f->status);
    delete f;
}

unsigned grid_of(uint64_t B) { return (unsigned)((B + kForWarps - 1) / kForWarps); }

template <typename KT>
int for_compress_t(const KT* keys, uint64_t n, cudaStream_t st, lc_for* f) {
    const uint64_t B = f->B;
    const size_t tmp_b = scan_tmp_bytes(B);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_base = 0, o_width = al(sizeof(KT) * B), o_words = o_width + al(B), o_tmp = o_words + al(4 * B);
    uint8_t* scratch = nullptr;
    if (cudaMalloc((void**)&scratch, o_tmp + tmp_b + 16) != cudaSuccess) return LC_ERR_NOMEM;
    KT* base = (KT*)(scratch + o_base);
    uint8_t* width = scratch + o_width;
    uint32_t* words = (uint32_t*)(scratch + o_words);
    int rc = LC_OK;
    {
        KTime kt("for_width", st);
        for_width_kernel<KT><<<grid_of(B), kForThreads, 0, st>>>(keys, n, B, base, width, words, f->status);
    }
    note_launch();
    rc = cuda_status(cudaGetLastError());
    if (!rc) rc = scan_exclusive(words, f->woff, B, ScanOp::Identity, scratch + o_tmp, tmp_b, st);
    uint64_t W = 0;
    uint32_t h_status = 0;
    if (!rc) rc = cuda_status(cudaMemcpyAsync(&W, f->woff + B, 8, cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaMemcpyAsync(&h_status, f->status, 4, cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    if (!rc && (h_status & kStUnsorted)) rc = LC_ERR_UNSORTED;
    if (!rc) {
        f->W = W;
        for_layout(f);
        if (cudaMalloc((void**)&f->blob, f->total) != cudaSuccess) {
            f->blob = nullptr;
            rc = LC_ERR_NOMEM;
        }
    }
    if (!rc) {
        uint8_t hdr[32];
        std::memset(hdr, 0, sizeof hdr);
        std::memcpy(hdr, "FOR1", 4);
        std::memcpy(hdr + 4, &f->key_bytes, 4);
        std::memcpy(hdr + 8, &f->N, 8);
        std::memcpy(hdr + 16, &f->B, 8);
        std::memcpy(hdr + 24, &f->W, 8);
        rc = cuda_status(cudaMemcpyAsync(f->blob, hdr, 32, cudaMemcpyHostToDevice, st));
        if (!rc) rc = cuda_status(cudaMemcpyAsync(f->blob + f->off_base, base, sizeof(KT) * B, cudaMemcpyDeviceToDevice, st));
        if (!rc) rc = cuda_status(cudaMemcpyAsync(f->blob + f->off_width, width, B, cudaMemcpyDeviceToDevice, st));
        if (!rc) {
            for_zero_kernel<<<1, 256, 0, st>>>(f->blob, f->off_base + sizeof(KT) * B, f->off_width,
                                               f->off_width + B, f->off_payload);
            note_launch();
            KTime kt("for_pack", st);
            for_pack_kernel<KT><<<grid_of(B), kForThreads, 0, st>>>(keys, n, B, width, f->woff,
                                                                   (uint32_t*)(f->blob + f->off_payload));
            note_launch();
            rc = cuda_status(cudaGetLastError());
        }
        if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    }
    cudaFree(scratch);
    return rc;
}

}  // namespace
}  // namespace lcx

using namespace lcx;

extern "C" {

int lc_for_compress(const void* keys_dev, uint64_t n, int key_bytes, void* stream, lc_for** out) {
    if (!out || (key_bytes != 4 && key_bytes != 8) || (n && !keys_dev)) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    lc_for* f = new (std::nothrow) lc_for();
    if (!f) return LC_ERR_NOMEM;
    cudaGetDevice(&f->device);
    f->key_bytes = (uint32_t)key_bytes;
    f->N = n;
    f->B = (n + kForBlock - 1) / kForBlock;
    int rc = LC_OK;
    if (cudaMalloc((void**)&f->woff, 8 * (f->B + 1)) != cudaSuccess) rc = LC_ERR_NOMEM;
    if (!rc && cudaMalloc((void**)&f->status, 16) != cudaSuccess) rc = LC_ERR_NOMEM;
    if (!rc) rc = cuda_status(cudaMemsetAsync(f->status, 0, 16, st));
    if (!rc && n == 0) {
        f->W = 0;
        for_layout(f);
        if (cudaMalloc((void**)&f->blob, f->total) != cudaSuccess) {
            f->blob = nullptr;
            rc = LC_ERR_NOMEM;
        } else {
            uint8_t hdr[32];
            std::memset(hdr, 0, sizeof hdr);
            std::memcpy(hdr, "FOR1", 4);
            std::memcpy(hdr + 4, &f->key_bytes, 4);
            rc = cuda_status(cudaMemcpyAsync(f->blob, hdr, 32, cudaMemcpyHostToDevice, st));
            if (!rc) rc = cuda_status(cudaMemsetAsync(f->woff, 0, 8, st));
            if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
        }
    } else if (!rc) {
        rc = key_bytes == 4 ? for_compress_t<uint32_t>((const uint32_t*)keys_dev, n, st, f)
                            : for_compress_t<uint64_t>((const uint64_t*)keys_dev, n, st, f);
    }
    if (rc) {
        for_free(f);
        return rc;
    }
    *out = f;
    return LC_OK;
}

int lc_for_decode(const lc_for* f, void* out_dev, void* stream) {
    if (!f || (f->N && !out_dev)) return LC_ERR_INVALID_ARG;
    if (f->N == 0) return LC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    {
        KTime kt("for_decode", st);
        if (f->key_bytes == 4)
            for_decode_kernel<uint32_t><<<grid_of(f->B), kForThreads, 0, st>>>(
                f->blob, f->off_base, f->off_width, f->off_payload, f->N, f->B, f->woff, (uint32_t*)out_dev);
        else
            for_decode_kernel<uint64_t><<<grid_of(f->B), kForThreads, 0, st>>>(
                f->blob, f->off_base, f->off_width, f->off_payload, f->N, f->B, f->woff, (uint64_t*)out_dev);
    }
    note_launch();
    return cuda_status(cudaGetLastError());
}

int lc_for_size(const lc_for* f, uint64_t* bytes) {
    if (!f || !bytes) return LC_ERR_INVALID_ARG;
    *bytes = f->total;
    return LC_OK;
}

int lc_for_serialize(const lc_for* f, void* host, uint64_t cap, uint64_t* len) {
    if (!f || !len) return LC_ERR_INVALID_ARG;
    *len = f->total;
    if (!host || cap < f->total) return LC_ERR_INVALID_ARG;
    return cuda_status(cudaMemcpy(host, f->blob, f->total, cudaMemcpyDeviceToHost));
}

void lc_for_free(lc_for* f) { for_free(f); }

}  // extern "C"
