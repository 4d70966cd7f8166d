// lc_math.cuh -- exact integer arithmetic of the anchored fixed-point eps-PLA
// on the device (Def. 2, Eq. (1) of arXiv 2412.10770 with an int64 Q32 slope).
#pragma once

#include <cstdint>

namespace lcx {

// floor(M * d / 2^32) for an int64 Q32 slope M and 0 <= d < 2^32: the integer
// part of the anchored line at distance d from its anchor.  Exact: M = hi*2^32
// + lo with lo unsigned, so the product splits into hi*d (exact) plus the high
// word of lo*d.
__device__ __forceinline__ int64_t line_at(int64_t M, uint32_t d) {
    int32_t hi = (int32_t)(M >> 32);
    uint32_t lo = (uint32_t)M;
    return (int64_t)hi * (int64_t)d + (int64_t)__umulhi(lo, d);
}

// floor(n / d) for n < 2^49 and 2 <= d < 2^16, given m = ceil(2^64 / d).
// n*m/2^64 = n/d + n*e/(d*2^64) with 0 <= e < d, so the estimate is floor(n/d)
// or one more; one comparison corrects it.
__device__ __forceinline__ uint64_t udiv_magic(uint64_t n, uint32_t d, uint64_t m) {
    uint64_t q = __umul64hi(n, m);
    if (q * d > n) --q;
    return q;
}

// ceil(X * 2^32 / d) for |X| < 2^49 and 1 <= d < 2^16, when the result fits in
// int64 (callers only ask for cone bounds that do).
__device__ __forceinline__ int64_t ceil_q32(int64_t X, uint32_t d, const uint64_t* __restrict__ magic) {
    if (d == 1) return (int64_t)((uint64_t)X << 32);
    uint64_t m = __ldg(magic + d);
    if (X >= 0) {
        uint64_t a = (uint64_t)X;
        uint64_t q1 = udiv_magic(a, d, m);
        uint64_t r1 = a - q1 * d;
        uint64_t q2 = udiv_magic((r1 << 32) + d - 1, d, m);
        return (int64_t)((q1 << 32) + q2);
    }
    uint64_t a = (uint64_t)(-X);
    uint64_t q1 = udiv_magic(a, d, m);
    uint64_t r1 = a - q1 * d;
    uint64_t q2 = udiv_magic(r1 << 32, d, m);
    return -(int64_t)((q1 << 32) + q2);
}

// One step of the shrinking cone: can key i (d = i - s >= 1, D = K[i] - K[s])
// join the segment anchored at s whose admissible Q32 slopes are [LO, HI]?
// The integer slopes that keep |D - floor(M d / 2^32)| <= eps are exactly
// [ceil((D-eps) 2^32/d), ceil((D+eps+1) 2^32/d) - 1]; the key joins iff that
// interval meets [LO, HI].  Both tests reduce to the line values at d of the
// two cone edges, so no division is needed unless an edge moves.
__device__ __forceinline__ bool cone_step(uint64_t D, uint32_t d, int64_t eps, int64_t& LO, int64_t& HI,
                                          const uint64_t* __restrict__ magic) {
    if (D >= (1ull << 48)) return false;  // slope above 2^31 per key: no int64 Q32 slope fits
    int64_t dlo = (int64_t)D - eps, dhi = (int64_t)D + eps;
    int64_t pl = line_at(LO, d), ph = line_at(HI, d);
    if (pl > dhi || ph < dlo) return false;
    if (pl < dlo) LO = ceil_q32(dlo, d, magic);
    if (ph > dhi) HI = ceil_q32(dhi + 1, d, magic) - 1;
    return true;
}

// The same cone without division.  Key t admits the real Q32 slopes in
// [2^32 (D_t - eps)/d_t, 2^32 (D_t + eps + 1)/d_t); the integer cone of a run
// of keys is non-empty iff ceil(max lower) < ceil(min upper).  Both extremes
// are fractions x/e and y/f with e, f < 2^16, so their gap, when positive, is
// 2^32 (y e - x f)/(e f) >= 2^32/(e f) > 1: the integer cone is non-empty iff
// x/e < y/f as fractions.  The int64 cap on the slope is the upper fraction
// 2^31/1 a fresh cone starts from.  State: max lower x/e (X, E) and min upper
// y/f (Y, F).  Returns false (state unchanged) when key (D, d) empties it.
struct Frac {
    int64_t X;   // max (D - eps) over keys, as X / E
    uint32_t E;
    uint64_t Y;  // min (D + eps + 1), as Y / F
    uint32_t F;
};

__device__ __forceinline__ Frac frac_open() { return Frac{-(1ll << 31), 1u, 1ull << 31, 1u}; }

// x1/e1 > x2/e2 for |x| < 2^47 and 0 < e < 2^16 (no overflow).
__device__ __forceinline__ bool frac_gt(int64_t x1, uint32_t e1, int64_t x2, uint32_t e2) {
    return x1 * (int64_t)e2 > x2 * (int64_t)e1;
}

__device__ __forceinline__ bool frac_ok(const Frac& c) {
    return c.X < 0 || (uint64_t)c.X * c.F < c.Y * c.E;
}

__device__ __forceinline__ bool frac_step(uint64_t D, uint32_t d, int64_t eps, Frac& c) {
    if (D >= ((uint64_t)d << 31) + (uint64_t)eps) return false;  // lower bound at or above the int64 cap
    const int64_t xl = (int64_t)D - eps;
    const uint64_t yh = D + (uint64_t)eps + 1;
    Frac n = c;
    if (frac_gt(xl, d, c.X, c.E)) { n.X = xl; n.E = d; }
    if (yh * (uint64_t)c.F < c.Y * (uint64_t)d) { n.Y = yh; n.F = d; }
    if (!frac_ok(n)) return false;
    c = n;
    return true;
}

// The slope of a closed segment from its cone: the floor midpoint of
// [LO, HI] with LO = ceil(2^32 X/E) and HI = ceil(2^32 Y/F) - 1, capped at
// INT64_MAX (the fraction 2^31/1 or above).
__device__ __forceinline__ int64_t frac_slope(const Frac& c, const uint64_t* __restrict__ magic) {
    const int64_t LO = ceil_q32(c.X, c.E, magic);
    const int64_t HI = c.Y >= ((uint64_t)c.F << 31) ? INT64_MAX : ceil_q32((int64_t)c.Y, c.F, magic) - 1;
    return LO + (int64_t)(((uint64_t)HI - (uint64_t)LO) >> 1);
}

__device__ __forceinline__ uint32_t zigzag32(int64_t r) {
    return (uint32_t)(((uint64_t)r << 1) ^ (uint64_t)(r >> 63));
}

__device__ __forceinline__ int32_t unzigzag32(uint32_t z) {
    return (int32_t)((z >> 1) ^ (0u - (z & 1u)));
}

// Low w bits of the 32-bit field starting at bit `sh` of the pair (lo, hi),
// 0 <= w <= 32.
__device__ __forceinline__ uint32_t extract_bits(uint32_t lo, uint32_t hi, uint32_t sh, uint32_t w) {
    uint32_t v = __funnelshift_r(lo, hi, sh);
    uint32_t r;
    asm("bfe.u32 %0, %1, 0, %2;" : "=r"(r) : "r"(v), "r"(w));
    return r;
}

}  // namespace lcx
