// rs_numeric.cuh -- exact integer and double-float arithmetic for RSI scoring.
//
// GB300 (sm_103a) executes FP64 at 1/64 of its FP32 rate, so the per-edge and
// per-column arithmetic of the score runs on the integer and FP32 pipes:
//
//  * entropy numerators E = Y log2 Y - sum_j f_j log2 f_j (Eq. H_optimal of
//    Sec. IV-B, with Y = T - f_i) are exact 128-bit integer sums of a log2
//    table LG[f] = round(log2(f) 2^58); the only error is the table's
//    rounding, |dE| <= Y 2^-58, and E >= log2 Y + 1.44 whenever two or more
//    communities remain, so E/Y keeps ~1e-14 relative accuracy for Y <= 1e5;
//  * quotients, cube roots and products use double-float numbers (an
//    unevaluated sum hi + lo of two floats, ~2^-48 relative; Dekker 1971,
//    "A floating-point technique for extending the available precision");
//  * every sum of terms is accumulated in 128-bit fixed point (2^-64 lsb), so
//    atomics commute and results are bit-identical whatever the schedule.
#pragma once
#include <stdint.h>

namespace rs {

typedef unsigned __int128 u128;

constexpr int kLogFrac = 58;      // LG[f] = round(log2(f) * 2^58)
constexpr int kSFrac = 52;        // node scalar s_v stored as round(s_v * 2^52)
constexpr int kAccFrac = 64;      // accumulators: 2^-64 lsb

// ---- double-float ----------------------------------------------------------

struct df { float hi, lo; };

__device__ __forceinline__ df df_make(float a) { return df{a, 0.0f}; }

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {   // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}
__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return df{p, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return quick_two_sum(p.hi, p.lo);
}
// a / y for an integer 1 <= y < 2^24 (exact as a float)
__device__ __forceinline__ df df_div_u32(df a, uint32_t y) {
    float fy = (float)y;
    float r = __frcp_rn(fy);
    float q1 = __fmul_rn(a.hi, r);
    df p = two_prod(q1, fy);
    float rem = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);
    float q2 = __fmul_rn(rem, r);
    df q = quick_two_sum(q1, q2);
    // one more correction step: residual of q against a
    df back = df_mul_f(q, fy);
    float rem2 = __fadd_rn(__fsub_rn(a.hi, back.hi), __fsub_rn(a.lo, back.lo));
    return df_add(q, df_make(__fmul_rn(rem2, r)));
}
// a^(1/3), a >= 0: float seed, one Newton step evaluated in double-float
__device__ __forceinline__ df df_cbrt(df a) {
    if (!(a.hi > 0.0f)) return df{0.0f, 0.0f};
    float y = cbrtf(a.hi);
    df y2 = two_prod(y, y);                       // y^2 exactly
    df y3 = df_mul_f(y2, y);                      // y^3
    df r = df_add(a, df{-y3.hi, -y3.lo});         // a - y^3
    float c = __fmul_rn(r.hi, __frcp_rn(__fmul_rn(3.0f, y2.hi)));
    return two_sum(y, c);
}
__device__ __forceinline__ bool df_less(df a, df b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ df df_max(df a, df b) { return df_less(a, b) ? b : a; }

// ---- conversions -------------------------------------------------------------

// 2^e as a float for -126 <= e <= 127 (exact)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// x * 2^e as double-float, keeping the top 48 significant bits of x
// (the exponents reached by the score stay inside the normal float range)
__device__ __forceinline__ df df_from_u128(u128 x, int e) {
    if (x == 0) return df{0.0f, 0.0f};
    uint64_t h = (uint64_t)(x >> 64);
    int lz = h ? __clzll((long long)h) : 64 + __clzll((long long)(uint64_t)x);
    int top = 127 - lz;                           // index of the leading bit
    int sh = top - 47;                            // keep bits [top-47, top]
    uint64_t m48 = sh >= 0 ? (uint64_t)(x >> sh) : (uint64_t)x << (-sh);
    uint32_t mh = (uint32_t)(m48 >> 24), ml = (uint32_t)(m48 & 0xFFFFFFu);
    float hi = __fmul_rn((float)mh, pow2f(sh + 24 + e));
    float lo = __fmul_rn((float)ml, pow2f(sh + e));
    return quick_two_sum(hi, lo);
}
__device__ __forceinline__ df df_from_u64(uint64_t x, int e) { return df_from_u128((u128)x, e); }

// f * 2^frac truncated toward zero, as a two's complement 128-bit integer (hi:lo), for
// a finite float f: its 24-bit significand shifted by the exponent, with 64-bit pieces
// (every score term keeps the shift below 128)
__device__ __forceinline__ void fixed_part(float f, int frac, uint64_t &lo, uint64_t &hi) {
    const uint32_t b = __float_as_uint(f);
    const int ex = (int)((b >> 23) & 0xFF);
    const uint32_t mant = (b & 0x7FFFFFu) | (ex ? 0x800000u : 0u);
    const int q = (ex ? ex - 150 : -149) + frac;
    uint64_t l, h;
    if (q >= 64) {
        l = 0;
        h = (uint64_t)mant << (q - 64);
    } else if (q > 0) {
        l = (uint64_t)mant << q;
        h = (uint64_t)mant >> (64 - q);
    } else {
        const int s = -q;                          // bits below 1 are dropped
        l = s < 32 ? (uint64_t)(mant >> s) : 0;
        h = 0;
    }
    if (b >> 31) {                                 // negative: the magnitude's two's complement
        l = ~l + 1;
        h = ~h + (l == 0 ? 1 : 0);
    }
    lo = l;
    hi = h;
}
// round-toward-zero of each part of a * 2^frac, summed, for a >= 0 as an unsigned
// 128-bit integer (0 when the sum is negative).  The usual case takes a short path with
// the same result: a.hi a positive normal float whose scaled significand ends below bit
// 64 (0 < qh < 64, which for 0 <= frac <= 64, the scales used, already makes a.hi
// positive, normal and finite), and a.lo at least 2^24 times smaller in exponent
// (el <= eh - 24, true of every normalised double-float).  Then a.hi's significand is
// shifted into place, and a.lo * 2^frac (exact: a power-of-two scaling) is converted to
// int64 with truncation toward zero, which is the magnitude's truncation with a.lo's sign
// (and 0 for a subnormal a.lo, below 2^-62 once scaled); ql <= qh - 24 < 40 keeps that
// value under 2^63.  Since |a.lo| < 2^(eh-150) = ulp(a.hi), |a.lo| 2^frac < 2^qh, at most
// 2^-23 of a.hi's part, so the sum is positive and below 2^88: no clamp is needed there.
__device__ __forceinline__ u128 df_to_fixed(df a, int frac) {
    const uint32_t bh = __float_as_uint(a.hi), bl = __float_as_uint(a.lo);
    const int eh = (int)(bh >> 23);                // with the sign bit: < 255 means a.hi >= 0, finite
    const int el = (int)((bl >> 23) & 0xFF);
    const int qh = eh - 150 + frac;
    if ((uint32_t)(qh - 1) < 63u && el + 24 <= eh) {
        const uint64_t mh = (uint64_t)((bh & 0x7FFFFFu) | 0x800000u);
        const uint64_t l = mh << qh, h = mh >> (64 - qh);
        const int64_t lp = __float2ll_rz(__fmul_rn(a.lo, pow2f(frac)));
        const uint64_t l2 = l + (uint64_t)lp;
        const uint64_t h2 = h + (lp < 0 ? ~0ull : 0ull) + (l2 < l ? 1ull : 0ull);
        return ((u128)h2 << 64) | l2;
    }
    uint64_t l1, h1, l2, h2;
    fixed_part(a.hi, frac, l1, h1);
    fixed_part(a.lo, frac, l2, h2);
    const uint64_t lo = l1 + l2;
    const uint64_t hi = h1 + h2 + (lo < l1 ? 1 : 0);
    if ((int64_t)hi < 0) return 0;
    return ((u128)hi << 64) | lo;
}

// correctly rounded (nearest, ties to even) double of x * 2^e, x < 2^128, |e| moderate
__device__ __forceinline__ double u128_to_double(u128 x, int e) {
    if (x == 0) return 0.0;
    uint64_t h = (uint64_t)(x >> 64);
    int lz = h ? __clzll((long long)h) : 64 + __clzll((long long)(uint64_t)x);
    int top = 127 - lz;
    uint64_t mant;
    if (top <= 52) {
        mant = (uint64_t)x << (52 - top);
    } else {
        int sh = top - 52;
        mant = (uint64_t)(x >> sh);
        u128 rem = x & (((u128)1 << sh) - 1);
        u128 half = (u128)1 << (sh - 1);
        if (rem > half || (rem == half && (mant & 1))) {
            mant++;
            if (mant >> 53) { mant >>= 1; top++; }
        }
    }
    int exp2 = top + e;                            // value = 1.mant * 2^exp2
    int biased = exp2 + 1023;
    if (biased <= 0) return 0.0;                   // never reached for scores
    uint64_t bits = ((uint64_t)biased << 52) | (mant & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// ---- 128-bit accumulators -------------------------------------------------------

// acc[0] holds the low 64 bits, acc[1] the high 64 bits; concurrent adds commute
__device__ __forceinline__ void atomic_add_u128(unsigned long long *acc, u128 v) {
    unsigned long long lo = (unsigned long long)(uint64_t)v;
    unsigned long long hi = (unsigned long long)(uint64_t)(v >> 64);
    if (lo) {
        unsigned long long old = atomicAdd(acc, lo);
        if (old + lo < old) hi += 1ull;
    }
    if (hi) atomicAdd(acc + 1, hi);
}

// ---- warp reductions ---------------------------------------------------------------

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int m) {
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_xor_sync(0xFFFFFFFFu, lo, m);
    hi = __shfl_xor_sync(0xFFFFFFFFu, hi, m);
    return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
    for (int m = 16; m; m >>= 1) v += shfl_xor_u128(v, m);
    return v;
}
__device__ __forceinline__ df warp_max_df(df v) {
    for (int m = 16; m; m >>= 1) {
        df o{__shfl_xor_sync(0xFFFFFFFFu, v.hi, m), __shfl_xor_sync(0xFFFFFFFFu, v.lo, m)};
        v = df_max(v, o);
    }
    return v;
}

// ---- entropy weights (Eq. entropy / weight via Eq. H_optimal) ----------------------
//
// Row aggregates of node v over its neighbour communities: T = d(v), L = number
// of distinct communities, X = sum_c f_c LG[f_c] (exact).  The weight of column
// c with count f (f = 0 for a community absent from N(v)) is
//     w = H(L_c) |L_c|,  H(L_c) = E / Y,  Y = T - f,  E = Y LG[Y] - (X - f LG[f]),
// |L_c| = L - [f > 0], and w = 0 when |L_c| < 2.  Under the convention of Alg. 2
// (|L| = L_all - 1 for every column, also when c is absent from N(v)), which the
// table flags with LG[0] = 1, |L_c| = L - 1 for every column.
struct RowAgg {
    uint32_t T;      // degree
    uint32_t L;      // distinct communities among the neighbours
    u128 X;          // sum_c f_c * LG[f_c]
};

__device__ __forceinline__ df column_weight(const RowAgg &a, uint32_t f, const uint64_t *LG) {
    uint32_t drop = (f > 0 || (LG[0] & 1)) ? 1u : 0u;
    if (a.L < drop + 2) return df{0.0f, 0.0f};
    uint32_t Lc = a.L - drop;
    uint32_t Y = a.T - f;
    u128 rest = a.X - (u128)f * LG[f];
    u128 yy = (u128)Y * LG[Y];
    u128 E = yy > rest ? yy - rest : (u128)0;
    df H = df_div_u32(df_from_u128(E, -kLogFrac), Y);
    return df_mul_f(H, (float)Lc);
}

}  // namespace rs
