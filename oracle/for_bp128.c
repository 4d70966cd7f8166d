/*
 * for_bp128.c -- plain CPU reference of the frame-of-reference delta
 * bit-packing baseline (blocks of 128 keys, format "FOR1").
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the tests, the smoke
 * check and the benchmark's CPU leg load it; the CUDA library never does, and
 * the two share no code.
 *
 * This codec is not the paper's method: it is one of the conventional
 * integer codecs the paper compares its learned compressor with (Sec. II-C,
 * Fig. 3a), used here as the GPU baseline of the scale sweep.  Definition:
 *   - blocks of 128 keys, B = ceil(N / 128), the last one ragged;
 *   - block b: base = K[128b]; gaps g_0 = 0, g_i = K[128b+i] - K[128b+i-1]
 *     for 128b + i < N, and g_i = 0 past the last key;
 *   - w_b = bit length of max_i g_i (0 if all are 0);
 *   - the 128 gaps at w_b bits each, gap i at bit i * w_b of the block's
 *     payload, LSB-first in little-endian 32-bit words; block b occupies
 *     4 w_b words starting at word 4 (w_0 + ... + w_{b-1}).
 * Bytes: header 32 ("FOR1", key_bytes u32, N u64, B u64, W u64), block_base
 * (key_bytes x B), block_width (u8 x B), payload (u32 x W); every array starts
 * 16-byte aligned and padding bytes are 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "lc_oracle.h"

static uint64_t fo_pad16(uint64_t x) { return (x + 15u) & ~(uint64_t)15u; }

static void fo_put(uint8_t* p, uint64_t v, int bytes)
{
    for (int i = 0; i < bytes; ++i) p[i] = (uint8_t)(v >> (8 * i));
}

static uint64_t fo_get(const uint8_t* p, int bytes)
{
    uint64_t v = 0;
    for (int i = 0; i < bytes; ++i) v |= (uint64_t)p[i] << (8 * i);
    return v;
}

static unsigned fo_bitlen(uint64_t x)
{
    unsigned b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

static uint64_t fo_gap(const uint8_t* keys, int kb, uint64_t n, uint64_t b, unsigned i)
{
    const uint64_t k = 128 * b + i;
    if (i == 0 || k >= n) return 0;
    return fo_get(keys + kb * k, kb) - fo_get(keys + kb * (k - 1), kb);
}

int lco_for_compress(const void* keys_v, uint64_t n, int kb, uint8_t** blob, uint64_t* len)
{
    if (!blob || !len || (kb != 4 && kb != 8) || (n && !keys_v)) return LCO_ERR_INVALID_ARG;
    const uint8_t* keys = (const uint8_t*)keys_v;
    for (uint64_t i = 1; i < n; ++i)
        if (fo_get(keys + kb * i, kb) < fo_get(keys + kb * (i - 1), kb)) return LCO_ERR_UNSORTED;
    const uint64_t B = (n + 127) / 128;
    uint64_t W = 0;
    unsigned* width = (unsigned*)calloc(B ? B : 1, sizeof(unsigned));
    if (!width) return LCO_ERR_NOMEM;
    for (uint64_t b = 0; b < B; ++b) {
        uint64_t m = 0;
        for (unsigned i = 0; i < 128; ++i) {
            const uint64_t g = fo_gap(keys, kb, n, b, i);
            if (g > m) m = g;
        }
        width[b] = fo_bitlen(m);
        W += 4 * (uint64_t)width[b];
    }
    const uint64_t off_base = 32, off_width = off_base + fo_pad16((uint64_t)kb * B);
    const uint64_t off_pay = off_width + fo_pad16(B), total = off_pay + 4 * W;
    uint8_t* out = (uint8_t*)calloc(total, 1);
    if (!out) {
        free(width);
        return LCO_ERR_NOMEM;
    }
    memcpy(out, "FOR1", 4);
    fo_put(out + 4, (uint64_t)kb, 4);
    fo_put(out + 8, n, 8);
    fo_put(out + 16, B, 8);
    fo_put(out + 24, W, 8);
    uint64_t word = 0;
    for (uint64_t b = 0; b < B; ++b) {
        fo_put(out + off_base + kb * b, fo_get(keys + kb * 128 * b, kb), kb);
        out[off_width + b] = (uint8_t)width[b];
        const unsigned w = width[b];
        uint8_t* pay = out + off_pay + 4 * word;
        for (unsigned i = 0; i < 128; ++i) {
            const uint64_t g = fo_gap(keys, kb, n, b, i);
            for (unsigned t = 0; t < w; ++t) {
                const uint64_t bit = (uint64_t)i * w + t; /* bit of the block payload */
                if ((g >> t) & 1u) pay[bit / 8] |= (uint8_t)(1u << (bit % 8));
            }
        }
        word += 4 * (uint64_t)w;
    }
    free(width);
    *blob = out;
    *len = total;
    return LCO_OK;
}

int lco_for_decode(const uint8_t* blob, uint64_t len, void* out_v)
{
    if (!blob || len < 32 || memcmp(blob, "FOR1", 4) != 0) return LCO_ERR_CORRUPT;
    const int kb = (int)fo_get(blob + 4, 4);
    const uint64_t n = fo_get(blob + 8, 8), B = fo_get(blob + 16, 8), W = fo_get(blob + 24, 8);
    if ((kb != 4 && kb != 8) || B != (n + 127) / 128) return LCO_ERR_CORRUPT;
    const uint64_t off_base = 32, off_width = off_base + fo_pad16((uint64_t)kb * B);
    const uint64_t off_pay = off_width + fo_pad16(B);
    if (len != off_pay + 4 * W) return LCO_ERR_CORRUPT;
    uint8_t* out = (uint8_t*)out_v;
    uint64_t word = 0;
    for (uint64_t b = 0; b < B; ++b) {
        const unsigned w = blob[off_width + b];
        if (w > 8u * (unsigned)kb || word + 4 * (uint64_t)w > W) return LCO_ERR_CORRUPT;
        const uint8_t* pay = blob + off_pay + 4 * word;
        uint64_t key = fo_get(blob + off_base + kb * b, kb);
        for (unsigned i = 0; i < 128 && 128 * b + i < n; ++i) {
            uint64_t g = 0;
            for (unsigned t = 0; t < w; ++t) {
                const uint64_t bit = (uint64_t)i * w + t;
                g |= (uint64_t)((pay[bit / 8] >> (bit % 8)) & 1u) << t;
            }
            key += g;
            fo_put(out + kb * (128 * b + i), key, kb);
        }
        word += 4 * (uint64_t)w;
    }
    return word == W ? LCO_OK : LCO_ERR_CORRUPT;
}
