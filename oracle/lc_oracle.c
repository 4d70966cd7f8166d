/*
 * lc_oracle.c -- plain CPU oracle of the learned compressor (arXiv 2412.10770).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Written for
 * obviousness, not speed: exact 128-bit integer arithmetic, one key at a
 * time, one bit at a time.  The definitions it follows and the byte format it
 * writes are spelled out in lc_oracle.h.
 */
#include "lc_oracle.h"

#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

static const i128 TWO32 = (i128)1 << 32;

/* ---------------------------------------------------------------- helpers */

static i128 floor_div(i128 a, i128 b) /* b > 0 */
{
    i128 q = a / b;
    if (a % b != 0 && a < 0) q -= 1;
    return q;
}

static i128 ceil_div(i128 a, i128 b) /* b > 0 */
{
    i128 q = a / b;
    if (a % b != 0 && a > 0) q += 1;
    return q;
}

static uint64_t pad16(uint64_t x) { return (x + 15u) & ~(uint64_t)15u; }

static void put_le(uint8_t* p, uint64_t v, int bytes)
{
    for (int b = 0; b < bytes; b++) p[b] = (uint8_t)(v >> (8 * b));
}

static uint64_t get_le(const uint8_t* p, int bytes)
{
    uint64_t v = 0;
    for (int b = 0; b < bytes; b++) v |= (uint64_t)p[b] << (8 * b);
    return v;
}

static unsigned bit_length(uint64_t x)
{
    unsigned n = 0;
    while (x) { n++; x >>= 1; }
    return n;
}

static uint64_t zigzag(int64_t r) { return r >= 0 ? (uint64_t)r * 2u : (uint64_t)(-(r + 1)) * 2u + 1u; }

static int64_t unzigzag(uint64_t z) { return (z & 1u) ? -(int64_t)(z >> 1) - 1 : (int64_t)(z >> 1); }

/* floor(M * d / 2^32): the integer part of segment j's line at distance d
 * from its anchor (Def. 2, Eq. (1), anchored fixed-point reading). */
static int64_t line_offset(int64_t M, uint64_t d)
{
    return (int64_t)floor_div((i128)M * (i128)d, TWO32);
}

static void put_bits(uint64_t* words, uint64_t pos, uint64_t value, unsigned w)
{
    for (unsigned b = 0; b < w; b++)
        if ((value >> b) & 1u) words[(pos + b) >> 6] |= (uint64_t)1 << ((pos + b) & 63u);
}

static uint64_t get_bits(const uint8_t* payload, uint64_t pos, unsigned w)
{
    uint64_t v = 0;
    for (unsigned b = 0; b < w; b++) {
        uint64_t p = pos + b;
        uint64_t word = get_le(payload + 8 * (p >> 6), 8);
        v |= ((word >> (p & 63u)) & 1u) << b;
    }
    return v;
}

/* ---------------------------------------------------------------- encoder */

typedef struct {
    uint64_t start; /* absolute key index of the anchor s_j */
    uint64_t n;     /* keys in the segment */
    int64_t slope;  /* M_j (Q32) */
    uint32_t width; /* w_j */
    uint32_t bitoff;
} oseg;

typedef struct {
    oseg* v;
    uint64_t n, cap;
} segvec;

static int segvec_push(segvec* s, oseg x)
{
    if (s->n == s->cap) {
        uint64_t cap = s->cap ? 2 * s->cap : 1024;
        oseg* nv = (oseg*)realloc(s->v, cap * sizeof(oseg));
        if (!nv) return LCO_ERR_NOMEM;
        s->v = nv;
        s->cap = cap;
    }
    s->v[s->n++] = x;
    return LCO_OK;
}

/* Close segment [s, s+n) whose cone is [LO, HI]: pick its slope (floor
 * midpoint of the cone; 0 for a single key), then its residuals' width. */
static int close_segment(const uint64_t* K, uint64_t s, uint64_t n, i128 LO, i128 HI,
                         uint64_t eps, segvec* out)
{
    oseg g;
    g.start = s;
    g.n = n;
    g.slope = n == 1 ? 0 : (int64_t)(LO + ((HI - LO) >> 1));
    uint64_t zmax = 0;
    for (uint64_t t = 1; t < n; t++) {
        i128 D = (i128)(K[s + t] - K[s]);
        i128 r = D - (i128)line_offset(g.slope, t);
        if (r > (i128)eps || r < -(i128)eps) return LCO_ERR_INTERNAL; /* Def. 2 violated */
        uint64_t z = zigzag((int64_t)r);
        if (z > zmax) zmax = z;
    }
    g.width = bit_length(zmax);
    g.bitoff = 0;
    return segvec_push(out, g);
}

/* The integer Q32 slopes key i admits in the segment anchored at s:
 * [lo, hi] with D - eps <= floor(M d / 2^32) <= D + eps (Def. 2),
 * d = i - s, D = K[i] - K[s]. */
static void key_bounds(const uint64_t* K, uint64_t s, uint64_t i, uint64_t eps, i128* lo_out, i128* hi_out)
{
    i128 d = (i128)(i - s);
    i128 D = (i128)(K[i] - K[s]);
    i128 lo = ceil_div((D - (i128)eps) * TWO32, d);
    i128 hi = floor_div((D + (i128)eps + 1) * TWO32 - 1, d);
    *lo_out = lo;
    *hi_out = hi;
}

/* Greedy shrinking-cone eps-PLA over the keys K[b, e) of one chunk. */
static int fit_chunk(const uint64_t* K, uint64_t b, uint64_t e, uint64_t eps, segvec* out)
{
    uint64_t s = b;
    i128 LO = INT64_MIN, HI = INT64_MAX;
    for (uint64_t i = b + 1; i < e; i++) {
        i128 lo, hi;
        key_bounds(K, s, i, eps, &lo, &hi);
        i128 nlo = LO > lo ? LO : lo;
        i128 nhi = HI < hi ? HI : hi;
        if (nlo <= nhi) {
            LO = nlo;
            HI = nhi;
            continue;
        }
        int rc = close_segment(K, s, i - s, LO, HI, eps, out);
        if (rc) return rc;
        s = i;
        LO = INT64_MIN;
        HI = INT64_MAX;
    }
    return close_segment(K, s, e - s, LO, HI, eps, out);
}

/* The integer cone [LO, HI] of the keys K[s+1, s+n) anchored at s: the
 * intersection of every key's admissible Q32 slopes (Def. 2). */
static void cone_of(const uint64_t* K, uint64_t s, uint64_t n, uint64_t eps, i128* LO_out, i128* HI_out)
{
    i128 LO = INT64_MIN, HI = INT64_MAX;
    for (uint64_t i = s + 1; i < s + n; i++) {
        i128 lo, hi;
        key_bounds(K, s, i, eps, &lo, &hi);
        if (lo > LO) LO = lo;
        if (hi < HI) HI = hi;
    }
    *LO_out = LO;
    *HI_out = HI;
}

/* The greedy's next anchor from p inside the chunk [b, e): the first key that
 * empties the cone anchored at p, or e. */
static uint64_t greedy_next(const uint64_t* K, uint64_t p, uint64_t e, uint64_t eps)
{
    i128 LO = INT64_MIN, HI = INT64_MAX;
    for (uint64_t i = p + 1; i < e; i++) {
        i128 lo, hi;
        key_bounds(K, p, i, eps, &lo, &hi);
        if (lo > LO) LO = lo;
        if (hi < HI) HI = hi;
        if (LO > HI) return i;
    }
    return e;
}

#define JUMP_H 96u            /* segments of at most this many keys take part in the jump */
#define JUMP_LONG UINT64_MAX  /* the greedy segment from p has more than JUMP_H keys */

/* The "jump" fit of one chunk, aiming at Sec. II-A's objective (the fewest
 * segments, which O'Rourke's algorithm reaches for free lines) within anchored
 * segments that are greedy prefixes.  r(p) = the greedy's next anchor from p
 * when that segment has at most JUMP_H keys, else JUMP_LONG.  From the anchor
 * a, the segment ends at the position in (a, r(a)] whose own r reaches
 * farthest (JUMP_LONG counts as farthest; ties: the first such position): the
 * jump-game choice, optimal when every segment is short.  A segment from an
 * anchor with r(a) = JUMP_LONG is the greedy's long segment.  The chunk keeps
 * this segmentation only if it has fewer segments than the greedy's. */
static int fit_chunk_jump(const uint64_t* K, uint64_t b, uint64_t e, uint64_t eps, segvec* out)
{
    const uint64_t n = e - b;
    uint64_t* r = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!r) return LCO_ERR_NOMEM;
    for (uint64_t p = b; p < e; p++) {
        uint64_t nx = greedy_next(K, p, e, eps);
        r[p - b] = nx - p <= JUMP_H ? nx : JUMP_LONG;
    }
    int rc = LCO_OK;
    /* the jump segmentation into its own list first: the chunk keeps it only
     * if it has fewer segments than the greedy's (ties: the greedy) */
    segvec jump = {0, 0, 0};
    uint64_t a = b;
    while (a < e && !rc) {
        uint64_t nx;
        if (r[a - b] == JUMP_LONG) {
            nx = greedy_next(K, a, e, eps);
        } else if (r[a - b] == e) {
            nx = e;
        } else {
            uint64_t best = a + 1, bk = r[a + 1 - b];
            for (uint64_t q = a + 2; q <= r[a - b]; q++)
                if (r[q - b] > bk) {
                    bk = r[q - b];
                    best = q;
                }
            nx = best;
        }
        i128 LO, HI;
        cone_of(K, a, nx - a, eps, &LO, &HI);
        rc = close_segment(K, a, nx - a, LO, HI, eps, &jump);
        a = nx;
    }
    free(r);
    if (!rc) {
        const uint64_t n0 = out->n;
        rc = fit_chunk(K, b, e, eps, out);
        if (!rc && jump.n < out->n - n0) {
            out->n = n0;
            for (uint64_t j = 0; j < jump.n && !rc; j++) rc = segvec_push(out, jump.v[j]);
        }
    }
    free(jump.v);
    return rc;
}

typedef struct {
    uint64_t key_begin, key_end, eps;
} ochunk;

static int g_fit_jump = 0; /* encode(): 0 the greedy fit, 1 the jump fit */

/* Shared back end of both entry points: chunks -> segments -> bytes. */
static int encode(const uint64_t* K, uint64_t N, int kb, const ochunk* ch, uint64_t C,
                  int list_mode, uint32_t chunk_log2, uint64_t eps_hdr,
                  const uint64_t* list_begin, const uint64_t* list_chunk_begin,
                  const uint64_t* list_eps, const uint8_t* list_log2, uint64_t NL,
                  uint8_t** blob_out, uint64_t* len_out)
{
    int rc = LCO_OK;
    segvec segs = {0, 0, 0};
    uint64_t* csb = (uint64_t*)calloc(C + 1, sizeof(uint64_t));
    uint64_t* cwb = (uint64_t*)calloc(C + 1, sizeof(uint64_t));
    uint64_t* payload = NULL;
    uint8_t* blob = NULL;
    if (!csb || !cwb) { rc = LCO_ERR_NOMEM; goto done; }

    /* 1. fit every chunk, then lay out its residual bits */
    for (uint64_t c = 0; c < C; c++) {
        csb[c] = segs.n;
        rc = g_fit_jump ? fit_chunk_jump(K, ch[c].key_begin, ch[c].key_end, ch[c].eps, &segs)
                        : fit_chunk(K, ch[c].key_begin, ch[c].key_end, ch[c].eps, &segs);
        if (rc) goto done;
        uint64_t bits = 0;
        for (uint64_t j = csb[c]; j < segs.n; j++) {
            segs.v[j].bitoff = (uint32_t)bits;
            bits += (uint64_t)segs.v[j].width * (segs.v[j].n - 1);
        }
        uint64_t words = (bits + 63) / 64;
        words += words & 1u; /* even: 16-byte aligned chunk payloads */
        cwb[c + 1] = cwb[c] + words;
    }
    csb[C] = segs.n;
    uint64_t L = segs.n, W = cwb[C];

    /* 2. pack residuals */
    payload = (uint64_t*)calloc(W ? W : 1, sizeof(uint64_t));
    if (!payload) { rc = LCO_ERR_NOMEM; goto done; }
    for (uint64_t c = 0; c < C; c++) {
        for (uint64_t j = csb[c]; j < csb[c + 1]; j++) {
            const oseg* g = &segs.v[j];
            for (uint64_t t = 1; t < g->n; t++) {
                int64_t r = (int64_t)((i128)(K[g->start + t] - K[g->start]) -
                                      (i128)line_offset(g->slope, t));
                uint64_t pos = 64 * cwb[c] + g->bitoff + (uint64_t)g->width * (t - 1);
                put_bits(payload, pos, zigzag(r), g->width);
            }
        }
    }

    /* 3. serialize */
    uint64_t off = 64, o_lkb = 0, o_lcb = 0, o_leps = 0, o_llog = 0;
    if (list_mode) {
        o_lkb = off; off += pad16(8 * (NL + 1));
        o_lcb = off; off += pad16(8 * (NL + 1));
        o_leps = off; off += pad16(8 * NL);
        o_llog = off; off += pad16(NL);
    }
    uint64_t o_ckb = off; off += pad16(8 * (C + 1));
    uint64_t o_csb = off; off += pad16(8 * (C + 1));
    uint64_t o_cwb = off; off += pad16(8 * (C + 1));
    uint64_t o_icpt = off; off += pad16((uint64_t)kb * L);
    uint64_t o_slope = off; off += pad16(8 * L);
    uint64_t o_bitoff = off; off += pad16(4 * L);
    uint64_t o_start = off; off += pad16(2 * L);
    uint64_t o_width = off; off += pad16(L);
    uint64_t o_pay = off; off += 8 * W;
    uint64_t total = off;

    blob = (uint8_t*)calloc(total, 1);
    if (!blob) { rc = LCO_ERR_NOMEM; goto done; }
    memcpy(blob, "LCF1", 4);
    put_le(blob + 4, 1, 2);
    put_le(blob + 6, list_mode ? 1 : 0, 2);
    put_le(blob + 8, (uint64_t)kb, 4);
    put_le(blob + 12, chunk_log2, 4);
    put_le(blob + 16, N, 8);
    put_le(blob + 24, eps_hdr, 8);
    put_le(blob + 32, C, 8);
    put_le(blob + 40, L, 8);
    put_le(blob + 48, W, 8);
    put_le(blob + 56, NL, 8);
    if (list_mode) {
        for (uint64_t l = 0; l <= NL; l++) {
            put_le(blob + o_lkb + 8 * l, list_begin[l], 8);
            put_le(blob + o_lcb + 8 * l, list_chunk_begin[l], 8);
        }
        for (uint64_t l = 0; l < NL; l++) {
            put_le(blob + o_leps + 8 * l, list_eps[l], 8);
            blob[o_llog + l] = list_log2[l];
        }
    }
    for (uint64_t c = 0; c <= C; c++) {
        put_le(blob + o_ckb + 8 * c, c < C ? ch[c].key_begin : N, 8);
        put_le(blob + o_csb + 8 * c, csb[c], 8);
        put_le(blob + o_cwb + 8 * c, cwb[c], 8);
    }
    for (uint64_t c = 0; c < C; c++) {
        for (uint64_t j = csb[c]; j < csb[c + 1]; j++) {
            const oseg* g = &segs.v[j];
            put_le(blob + o_icpt + (uint64_t)kb * j, K[g->start], kb);
            put_le(blob + o_slope + 8 * j, (uint64_t)g->slope, 8);
            put_le(blob + o_bitoff + 4 * j, g->bitoff, 4);
            put_le(blob + o_start + 2 * j, g->start - ch[c].key_begin, 2);
            blob[o_width + j] = (uint8_t)g->width;
        }
    }
    for (uint64_t w = 0; w < W; w++) put_le(blob + o_pay + 8 * w, payload[w], 8);

    *blob_out = blob;
    *len_out = total;
    blob = NULL;
done:
    free(segs.v);
    free(csb);
    free(cwb);
    free(payload);
    free(blob);
    return rc;
}

static uint64_t* widen_keys(const void* keys, uint64_t n, int kb)
{
    uint64_t* K = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!K) return NULL;
    const uint8_t* p = (const uint8_t*)keys;
    for (uint64_t i = 0; i < n; i++) K[i] = get_le(p + (uint64_t)kb * i, kb);
    return K;
}

int lco_compress(const void* keys, uint64_t n, int key_bytes, uint64_t eps, int chunk_log2,
                 uint8_t** blob, uint64_t* len)
{
    if (!blob || !len || (n && !keys)) return LCO_ERR_INVALID_ARG;
    if (key_bytes != 4 && key_bytes != 8) return LCO_ERR_INVALID_ARG;
    if (eps > ((uint64_t)1 << 30)) return LCO_ERR_INVALID_ARG;
    if (chunk_log2 < 8 || chunk_log2 > 16) return LCO_ERR_INVALID_ARG;
    uint64_t* K = widen_keys(keys, n, key_bytes);
    if (!K) return LCO_ERR_NOMEM;
    for (uint64_t i = 1; i < n; i++)
        if (K[i] < K[i - 1]) { free(K); return LCO_ERR_UNSORTED; }
    uint64_t cs = (uint64_t)1 << chunk_log2;
    uint64_t C = (n + cs - 1) / cs;
    ochunk* ch = (ochunk*)malloc((C ? C : 1) * sizeof(ochunk));
    if (!ch) { free(K); return LCO_ERR_NOMEM; }
    for (uint64_t c = 0; c < C; c++) {
        ch[c].key_begin = c * cs;
        ch[c].key_end = (c + 1) * cs < n ? (c + 1) * cs : n;
        ch[c].eps = eps;
    }
    int rc = encode(K, n, key_bytes, ch, C, 0, (uint32_t)chunk_log2, eps, NULL, NULL, NULL,
                    NULL, 0, blob, len);
    free(ch);
    free(K);
    return rc;
}

int lco_compress_jump(const void* keys, uint64_t n, int key_bytes, uint64_t eps, int chunk_log2,
                      uint8_t** blob, uint64_t* len)
{
    g_fit_jump = 1;
    int rc = lco_compress(keys, n, key_bytes, eps, chunk_log2, blob, len);
    g_fit_jump = 0;
    return rc;
}

int lco_compress_lists(const void* keys, const uint64_t* list_begin, uint64_t nlists,
                       int key_bytes, const uint64_t* eps, const uint8_t* chunk_log2,
                       uint8_t** blob, uint64_t* len)
{
    if (!blob || !len || !list_begin || (nlists && (!eps || !chunk_log2)))
        return LCO_ERR_INVALID_ARG;
    if (key_bytes != 4 && key_bytes != 8) return LCO_ERR_INVALID_ARG;
    if (list_begin[0] != 0) return LCO_ERR_INVALID_ARG;
    for (uint64_t l = 0; l < nlists; l++) {
        if (list_begin[l + 1] < list_begin[l]) return LCO_ERR_INVALID_ARG;
        if (eps[l] > ((uint64_t)1 << 30)) return LCO_ERR_INVALID_ARG;
        if (chunk_log2[l] < 8 || chunk_log2[l] > 16) return LCO_ERR_INVALID_ARG;
    }
    uint64_t n = list_begin[nlists];
    if (n && !keys) return LCO_ERR_INVALID_ARG;
    uint64_t* K = widen_keys(keys, n, key_bytes);
    if (!K) return LCO_ERR_NOMEM;
    uint64_t C = 0;
    for (uint64_t l = 0; l < nlists; l++) {
        for (uint64_t i = list_begin[l] + 1; i < list_begin[l + 1]; i++)
            if (K[i] < K[i - 1]) { free(K); return LCO_ERR_UNSORTED; }
        uint64_t cs = (uint64_t)1 << chunk_log2[l];
        C += (list_begin[l + 1] - list_begin[l] + cs - 1) / cs;
    }
    ochunk* ch = (ochunk*)malloc((C ? C : 1) * sizeof(ochunk));
    uint64_t* lcb = (uint64_t*)malloc((nlists + 1) * sizeof(uint64_t));
    if (!ch || !lcb) { free(ch); free(lcb); free(K); return LCO_ERR_NOMEM; }
    uint64_t c = 0;
    for (uint64_t l = 0; l < nlists; l++) {
        lcb[l] = c;
        uint64_t cs = (uint64_t)1 << chunk_log2[l];
        for (uint64_t b = list_begin[l]; b < list_begin[l + 1]; b += cs) {
            ch[c].key_begin = b;
            ch[c].key_end = b + cs < list_begin[l + 1] ? b + cs : list_begin[l + 1];
            ch[c].eps = eps[l];
            c++;
        }
    }
    lcb[nlists] = c;
    int rc = encode(K, n, key_bytes, ch, C, 1, 0, 0, list_begin, lcb, eps, chunk_log2, nlists,
                    blob, len);
    free(lcb);
    free(ch);
    free(K);
    return rc;
}

/* ---------------------------------------------------------------- decoder */

typedef struct {
    int kb, list_mode;
    uint32_t chunk_log2;
    uint64_t N, eps, C, L, W, NL;
    const uint8_t *lkb, *lcb, *leps, *llog, *ckb, *csb, *cwb;
    const uint8_t *icpt, *slope, *bitoff, *start, *width, *payload;
} oview;

static uint64_t U64(const uint8_t* a, uint64_t i) { return get_le(a + 8 * i, 8); }

static int zero_range(const uint8_t* b, uint64_t from, uint64_t to)
{
    for (uint64_t i = from; i < to; i++)
        if (b[i]) return 0;
    return 1;
}

/* Validate every structural fact of the format, then expose the arrays. */
static int parse(const uint8_t* blob, uint64_t len, oview* v)
{
    if (!blob || len < 64) return LCO_ERR_CORRUPT;
    if (memcmp(blob, "LCF1", 4) != 0) return LCO_ERR_CORRUPT;
    if (get_le(blob + 4, 2) != 1) return LCO_ERR_CORRUPT;
    uint64_t flags = get_le(blob + 6, 2);
    if (flags > 1) return LCO_ERR_CORRUPT;
    v->list_mode = (int)flags;
    v->kb = (int)get_le(blob + 8, 4);
    v->chunk_log2 = (uint32_t)get_le(blob + 12, 4);
    v->N = get_le(blob + 16, 8);
    v->eps = get_le(blob + 24, 8);
    v->C = get_le(blob + 32, 8);
    v->L = get_le(blob + 40, 8);
    v->W = get_le(blob + 48, 8);
    v->NL = get_le(blob + 56, 8);
    if (v->kb != 4 && v->kb != 8) return LCO_ERR_CORRUPT;
    const uint64_t big = (uint64_t)1 << 40;
    if (v->N > big || v->C > big || v->L > big || v->W > big || v->NL > big) return LCO_ERR_CORRUPT;
    if (v->list_mode) {
        if (v->chunk_log2 != 0 || v->eps != 0) return LCO_ERR_CORRUPT;
    } else {
        if (v->chunk_log2 < 8 || v->chunk_log2 > 16) return LCO_ERR_CORRUPT;
        if (v->eps > ((uint64_t)1 << 30) || v->NL != 0) return LCO_ERR_CORRUPT;
    }
    uint64_t off = 64, prev_end = 64;
    uint64_t o[13];
    uint64_t sz[13] = {
        v->list_mode ? 8 * (v->NL + 1) : 0, v->list_mode ? 8 * (v->NL + 1) : 0,
        v->list_mode ? 8 * v->NL : 0,       v->list_mode ? v->NL : 0,
        8 * (v->C + 1), 8 * (v->C + 1), 8 * (v->C + 1),
        (uint64_t)v->kb * v->L, 8 * v->L, 4 * v->L, 2 * v->L, v->L, 8 * v->W};
    for (int a = 0; a < 13; a++) {
        if (a < 4 && !v->list_mode) { o[a] = 0; continue; }
        o[a] = off;
        if (off > len || !zero_range(blob, prev_end, off < len ? off : len)) return LCO_ERR_CORRUPT;
        prev_end = off + sz[a];
        off += a == 12 ? sz[a] : pad16(sz[a]);
    }
    if (off != len) return LCO_ERR_CORRUPT;
    v->lkb = blob + o[0]; v->lcb = blob + o[1]; v->leps = blob + o[2]; v->llog = blob + o[3];
    v->ckb = blob + o[4]; v->csb = blob + o[5]; v->cwb = blob + o[6];
    v->icpt = blob + o[7]; v->slope = blob + o[8]; v->bitoff = blob + o[9];
    v->start = blob + o[10]; v->width = blob + o[11]; v->payload = blob + o[12];

    /* chunk directory */
    if (U64(v->ckb, 0) != 0 || U64(v->csb, 0) != 0 || U64(v->cwb, 0) != 0) return LCO_ERR_CORRUPT;
    if (U64(v->ckb, v->C) != v->N || U64(v->csb, v->C) != v->L || U64(v->cwb, v->C) != v->W)
        return LCO_ERR_CORRUPT;
    for (uint64_t c = 0; c < v->C; c++) {
        uint64_t kb0 = U64(v->ckb, c), kb1 = U64(v->ckb, c + 1);
        uint64_t s0 = U64(v->csb, c), s1 = U64(v->csb, c + 1);
        uint64_t w0 = U64(v->cwb, c), w1 = U64(v->cwb, c + 1);
        if (kb1 <= kb0 || kb1 - kb0 > 65536 || s1 <= s0 || s1 > v->L || w1 < w0 || ((w1 - w0) & 1u))
            return LCO_ERR_CORRUPT;
        uint64_t n_c = kb1 - kb0, bits = 0;
        for (uint64_t j = s0; j < s1; j++) {
            uint64_t st = get_le(v->start + 2 * j, 2);
            uint64_t en = j + 1 < s1 ? get_le(v->start + 2 * (j + 1), 2) : n_c;
            if ((j == s0 && st != 0) || en <= st || en > n_c) return LCO_ERR_CORRUPT;
            unsigned w = v->width[j];
            if (w > 32 || get_le(v->bitoff + 4 * j, 4) != bits) return LCO_ERR_CORRUPT;
            bits += (uint64_t)w * (en - st - 1);
        }
        uint64_t words = (bits + 63) / 64;
        words += words & 1u;
        if (w1 - w0 != words) return LCO_ERR_CORRUPT;
        /* pad bits after the chunk's last residual are 0 */
        for (uint64_t p = bits; p < 64 * words; p++)
            if (get_bits(v->payload, 64 * w0 + p, 1)) return LCO_ERR_CORRUPT;
    }
    /* chunk boundaries follow the chunking rule */
    if (!v->list_mode) {
        uint64_t cs = (uint64_t)1 << v->chunk_log2;
        if (v->C != (v->N + cs - 1) / cs) return LCO_ERR_CORRUPT;
        for (uint64_t c = 0; c < v->C; c++)
            if (U64(v->ckb, c) != c * cs) return LCO_ERR_CORRUPT;
    } else {
        if (U64(v->lkb, 0) != 0 || U64(v->lcb, 0) != 0) return LCO_ERR_CORRUPT;
        if (U64(v->lkb, v->NL) != v->N || U64(v->lcb, v->NL) != v->C) return LCO_ERR_CORRUPT;
        for (uint64_t l = 0; l < v->NL; l++) {
            uint64_t a = U64(v->lkb, l), b = U64(v->lkb, l + 1);
            uint64_t ca = U64(v->lcb, l), cb = U64(v->lcb, l + 1);
            unsigned lg = v->llog[l];
            if (b < a || cb < ca || lg < 8 || lg > 16 || U64(v->leps, l) > ((uint64_t)1 << 30))
                return LCO_ERR_CORRUPT;
            uint64_t cs = (uint64_t)1 << lg;
            if (cb - ca != (b - a + cs - 1) / cs) return LCO_ERR_CORRUPT;
            for (uint64_t c = ca; c < cb; c++)
                if (U64(v->ckb, c) != a + (c - ca) * cs) return LCO_ERR_CORRUPT;
        }
    }
    return LCO_OK;
}

static uint64_t icpt_of(const oview* v, uint64_t j) { return get_le(v->icpt + (uint64_t)v->kb * j, v->kb); }

/* Dec(K^c)[i] for key t of segment j of chunk c (Fig. 2 decoding stage:
 * K[i] = floor(f_j(i)) + Delta[i]). */
static uint64_t decode_one(const oview* v, uint64_t c, uint64_t j, uint64_t t)
{
    if (t == 0) return icpt_of(v, j);
    int64_t M = (int64_t)get_le(v->slope + 8 * j, 8);
    unsigned w = v->width[j];
    uint64_t pos = 64 * U64(v->cwb, c) + get_le(v->bitoff + 4 * j, 4) + (uint64_t)w * (t - 1);
    int64_t r = unzigzag(get_bits(v->payload, pos, w));
    i128 key = (i128)icpt_of(v, j) + (i128)line_offset(M, t) + (i128)r;
    return (uint64_t)key;
}

int lco_info(const uint8_t* blob, uint64_t len, uint64_t* n, int* key_bytes, uint64_t* chunks,
             uint64_t* segments, uint64_t* words)
{
    oview v;
    int rc = parse(blob, len, &v);
    if (rc) return rc;
    if (n) *n = v.N;
    if (key_bytes) *key_bytes = v.kb;
    if (chunks) *chunks = v.C;
    if (segments) *segments = v.L;
    if (words) *words = v.W;
    return LCO_OK;
}

int lco_decode(const uint8_t* blob, uint64_t len, void* out)
{
    oview v;
    int rc = parse(blob, len, &v);
    if (rc) return rc;
    if (v.N && !out) return LCO_ERR_INVALID_ARG;
    uint8_t* o = (uint8_t*)out;
    for (uint64_t c = 0; c < v.C; c++) {
        uint64_t base = U64(v.ckb, c), n_c = U64(v.ckb, c + 1) - base;
        uint64_t s0 = U64(v.csb, c), s1 = U64(v.csb, c + 1);
        for (uint64_t j = s0; j < s1; j++) {
            uint64_t st = get_le(v.start + 2 * j, 2);
            uint64_t en = j + 1 < s1 ? get_le(v.start + 2 * (j + 1), 2) : n_c;
            for (uint64_t t = 0; t < en - st; t++)
                put_le(o + (uint64_t)v.kb * (base + st + t), decode_one(&v, c, j, t), v.kb);
        }
    }
    return LCO_OK;
}

int lco_access(const uint8_t* blob, uint64_t len, const uint64_t* idx, uint64_t m, void* out)
{
    oview v;
    int rc = parse(blob, len, &v);
    if (rc) return rc;
    if (m && (!idx || !out)) return LCO_ERR_INVALID_ARG;
    for (uint64_t q = 0; q < m; q++) {
        uint64_t i = idx[q];
        if (i >= v.N) return LCO_ERR_OUT_OF_RANGE;
        /* chunk: last c with chunk_key_begin[c] <= i */
        uint64_t lo = 0, hi = v.C;
        while (hi - lo > 1) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (U64(v.ckb, mid) <= i) lo = mid; else hi = mid;
        }
        uint64_t c = lo, local = i - U64(v.ckb, c);
        /* segment: last j in the chunk with seg_start[j] <= local */
        uint64_t a = U64(v.csb, c), b = U64(v.csb, c + 1);
        while (b - a > 1) {
            uint64_t mid = a + (b - a) / 2;
            if (get_le(v.start + 2 * mid, 2) <= local) a = mid; else b = mid;
        }
        uint64_t t = local - get_le(v.start + 2 * a, 2);
        put_le((uint8_t*)out + (uint64_t)v.kb * q, decode_one(&v, c, a, t), v.kb);
    }
    return LCO_OK;
}

/* floor(f(i)) for every i in idx: the segments alone, no residual (Sec. III-C
 * approximate query processing; within eps of K[i] by Def. 2).  The segment
 * of i is found exactly as in lco_access. */
int lco_predict(const uint8_t* blob, uint64_t len, const uint64_t* idx, uint64_t m, void* out)
{
    oview v;
    int rc = parse(blob, len, &v);
    if (rc) return rc;
    if (m && (!idx || !out)) return LCO_ERR_INVALID_ARG;
    for (uint64_t q = 0; q < m; q++) {
        uint64_t i = idx[q];
        if (i >= v.N) return LCO_ERR_OUT_OF_RANGE;
        uint64_t lo = 0, hi = v.C;
        while (hi - lo > 1) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (U64(v.ckb, mid) <= i) lo = mid; else hi = mid;
        }
        uint64_t c = lo, local = i - U64(v.ckb, c);
        uint64_t a = U64(v.csb, c), b = U64(v.csb, c + 1);
        while (b - a > 1) {
            uint64_t mid = a + (b - a) / 2;
            if (get_le(v.start + 2 * mid, 2) <= local) a = mid; else b = mid;
        }
        uint64_t t = local - get_le(v.start + 2 * a, 2);
        int64_t M = (int64_t)get_le(v.slope + 8 * a, 8);
        i128 pred = (i128)icpt_of(&v, a) + (i128)(t ? line_offset(M, t) : 0);
        put_le((uint8_t*)out + (uint64_t)v.kb * q, (uint64_t)pred, v.kb);
    }
    return LCO_OK;
}

int lco_lower_bound(const uint8_t* blob, uint64_t len, const void* vals, uint64_t m, uint64_t* out)
{
    oview v;
    int rc = parse(blob, len, &v);
    if (rc) return rc;
    if (v.list_mode) return LCO_ERR_INVALID_ARG;
    if (m && (!vals || !out)) return LCO_ERR_INVALID_ARG;
    uint8_t* keys = (uint8_t*)malloc(v.N ? (size_t)(v.N * (uint64_t)v.kb) : 1);
    if (!keys) return LCO_ERR_NOMEM;
    rc = lco_decode(blob, len, keys);
    if (rc) { free(keys); return rc; }
    for (uint64_t q = 0; q < m; q++) {
        uint64_t x = get_le((const uint8_t*)vals + (uint64_t)v.kb * q, v.kb);
        uint64_t lo = 0, hi = v.N; /* first i in [lo, hi) with K[i] >= x */
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (get_le(keys + (uint64_t)v.kb * mid, v.kb) < x) lo = mid + 1; else hi = mid;
        }
        out[q] = lo;
    }
    free(keys);
    return LCO_OK;
}

void lco_free(void* p) { free(p); }
