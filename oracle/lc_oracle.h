/*
 * lc_oracle.h -- plain, slow CPU oracle of the learned compressor for sorted
 * integer keys (arXiv 2412.10770).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The product path (the CUDA
 * library and its Python binding) never links, loads or calls it, and the two
 * share no code.
 *
 * What the oracle computes, in the paper's notation:
 *   K[0..N)        sorted (non-decreasing) integer keys, 0-based (Fig. 2 uses
 *                  0-based indices; Def. 1 writes 1-based ones).
 *   f              an eps-PLA (Def. 2, Eq. (1)): segments (s_j, alpha_j, beta_j).
 *   Delta[i]       = K[i] - floor(f(i)), |Delta[i]| <= eps (Def. 2, Sec. II-A).
 *   K^c = (f, Delta), Dec(K^c)[i] = floor(f(i)) + Delta[i] = K[i] (Def. 1, Fig. 2).
 *
 * Readings fixed by this library (the paper leaves them open):
 *   - Model: anchored fixed-point lines.  beta_j = K[s_j]; alpha_j is an int64
 *     Q32 slope M_j; floor(f(i)) = K[s_j] + floor(M_j * (i - s_j) / 2^32), the
 *     product taken exactly (128-bit) and floored.
 *   - Fit: greedy shrinking cone inside fixed chunks of 2^b keys (b in [8,16]).
 *     From anchor s, key i (d = i - s, D = K[i] - K[s]) admits exactly the
 *     integer slopes M in [lo_i, hi_i] with
 *         lo_i = ceil((D - eps) * 2^32 / d),
 *         hi_i = floor(((D + eps + 1) * 2^32 - 1) / d),
 *     i.e. D - eps <= floor(M d / 2^32) <= D + eps.  The cone [LO, HI] starts
 *     at [INT64_MIN, INT64_MAX] and is intersected key by key; the first key
 *     that empties it starts the next segment.  A segment also ends at its
 *     chunk's end.
 *   - Slope: M = LO + floor((HI - LO) / 2) for segments of >= 2 keys, 0 for
 *     a single key.
 *   - Residual: Delta = D - floor(M d / 2^32) (exact), zigzag
 *     z = 2 Delta (Delta >= 0) or -2 Delta - 1 (Delta < 0).  Width of segment
 *     j: w_j = bit length of max z over its keys (0 if all are 0), which is
 *     <= ceil(log2(2 eps + 1)) (Sec. II-A).
 *   - Payload: the anchor's residual is always 0 and is not stored.  Residual
 *     t (1 <= t < n_j) of segment j is stored LSB-first at bit
 *     seg_bitoff_j + w_j (t - 1) of its chunk's payload; seg_bitoff is the
 *     running sum of w_j (n_j - 1) inside the chunk.  A chunk's payload spans
 *     an even number of 64-bit words (16-byte aligned), pad bits are 0.
 *
 * Serialized K^c, format "LCF1" (all little-endian; every array starts at a
 * 16-byte aligned offset; padding bytes are 0):
 *   header, 64 bytes:
 *     [0,4)  magic "LCF1"     [4,6) version u16 = 1   [6,8) flags u16 (bit 0: list mode)
 *     [8,12) key_bytes u32 (4|8)        [12,16) chunk_log2 u32 (0 in list mode)
 *     [16,24) N u64   [24,32) eps u64 (0 in list mode)   [32,40) C u64 (chunks)
 *     [40,48) L u64 (segments)   [48,56) W u64 (payload words)   [56,64) NL u64 (lists)
 *   list mode only:
 *     list_key_begin u64[NL+1], list_chunk_begin u64[NL+1], list_eps u64[NL],
 *     list_chunk_log2 u8[NL]
 *   always:
 *     chunk_key_begin u64[C+1], chunk_seg_begin u64[C+1], chunk_word_begin u64[C+1],
 *     seg_icpt key_bytes x L, seg_slope i64[L], seg_bitoff u32[L],
 *     seg_start u16[L] (chunk-relative), seg_width u8[L], payload u64[W]
 *   In list mode each list is its own column: chunks restart at each list's
 *   first key and use that list's eps and chunk_log2.
 */
#ifndef LC_ORACLE_H
#define LC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LCO_OK = 0,
    LCO_ERR_INVALID_ARG = -1,
    LCO_ERR_UNSORTED = -2,
    LCO_ERR_OUT_OF_RANGE = -3,
    LCO_ERR_NOMEM = -4,
    LCO_ERR_CORRUPT = -5,
    LCO_ERR_INTERNAL = -9
};

/* Compress one sorted column.  keys: n values of key_bytes (4 or 8) bytes,
 * host memory.  On success *blob is a malloc'ed buffer of *len bytes (free it
 * with lco_free).  eps <= 2^30, 8 <= chunk_log2 <= 16. */
int lco_compress(const void* keys, uint64_t n, int key_bytes, uint64_t eps,
                 int chunk_log2, uint8_t** blob, uint64_t* len);

/* The same with the "jump" fit in place of the greedy (fewest anchored
 * segments among greedy prefixes; optimal when no segment exceeds 96 keys,
 * Sec. II-A's objective): from anchor a, with r(p) = the greedy's next anchor
 * from p if that segment has <= 96 keys (else "long"), the next anchor is the
 * position in (a, r(a)] whose r reaches farthest (long = farthest; ties: the
 * first); an anchor whose own segment is long takes the greedy segment.  A
 * chunk keeps this segmentation only if it has fewer segments than the
 * greedy's (ties: the greedy).  Slopes, widths and bytes follow as for the
 * greedy.  Not thread-safe. */
int lco_compress_jump(const void* keys, uint64_t n, int key_bytes, uint64_t eps,
                      int chunk_log2, uint8_t** blob, uint64_t* len);

/* Compress nlists sorted lists stored back to back in keys.  list_begin has
 * nlists+1 entries (list l is keys[list_begin[l], list_begin[l+1])), eps and
 * chunk_log2 one entry per list. */
int lco_compress_lists(const void* keys, const uint64_t* list_begin, uint64_t nlists,
                       int key_bytes, const uint64_t* eps, const uint8_t* chunk_log2,
                       uint8_t** blob, uint64_t* len);

/* Read the header fields of a blob (after full validation). */
int lco_info(const uint8_t* blob, uint64_t len, uint64_t* n, int* key_bytes,
             uint64_t* chunks, uint64_t* segments, uint64_t* words);

/* Dec(K^c): all N keys, key_bytes each, into out. */
int lco_decode(const uint8_t* blob, uint64_t len, void* out);

/* K[idx[q]] for q < m into out (key_bytes each). */
int lco_access(const uint8_t* blob, uint64_t len, const uint64_t* idx, uint64_t m, void* out);

/* First i with K[i] >= v[q] (N if none), single-column blobs only.
 * v holds m values of key_bytes bytes. */
int lco_lower_bound(const uint8_t* blob, uint64_t len, const void* v, uint64_t m, uint64_t* out);

/* floor(f(idx[q])) from the segments alone (no residual), key_bytes each. */
int lco_predict(const uint8_t* blob, uint64_t len, const uint64_t* idx, uint64_t m, void* out);

void lco_free(void* p);

/* The frame-of-reference delta bit-packing baseline ("FOR1", blocks of 128
 * keys), defined in for_bp128.c: not the paper's method, the conventional
 * codec the scale sweep compares against.  Compress writes a malloc'ed blob
 * (lco_free); decode writes N keys. */
int lco_for_compress(const void* keys, uint64_t n, int key_bytes, uint8_t** blob, uint64_t* len);
int lco_for_decode(const uint8_t* blob, uint64_t len, void* out);

#ifdef __cplusplus
}
#endif

#endif /* LC_ORACLE_H */
