// numeric_host.cpp -- compiles the library's numerics header (rs_numeric.cuh) as host C++ and
// checks that df_to_fixed's short path gives the bits of its general path (each float part
// of the double-float truncated toward zero at the scale, the two summed, a negative sum
// clamped to 0) on random and edge-case inputs; with "accuracy N", bounds the relative errors
// of the double-float product, sum, quotient by an integer and cube root against long double.
// Test infrastructure: built and run by tests/test_numeric_host.py on the CPU.
//
// The device intrinsics the header uses are given their IEEE-754 meaning on the host (single
// precision, round to nearest; truncation toward zero for the float-to-int64 conversion);
// x86-64 and AArch64 evaluate float arithmetic in single precision.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

#define __device__
#define __forceinline__ inline
static inline uint32_t __float_as_uint(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }
static inline float __int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
static inline float __uint_as_float(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }
static inline double __longlong_as_double(long long x) { double d; std::memcpy(&d, &x, 8); return d; }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static inline float __frcp_rn(float a) { return 1.0f / a; }
static inline long long __float2ll_rz(float a) { return (long long)a; }
static inline int __clzll(long long x) { return x ? __builtin_clzll((unsigned long long)x) : 64; }
template <class T> static inline T __shfl_xor_sync(unsigned, T v, int) { return v; }   // not called here
static inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v) {   // not called here
    const unsigned long long o = *p;
    *p = o + v;
    return o;
}
#include "rs_numeric.cuh"

using rs::df;
using rs::u128;

// the general path of df_to_fixed, written from its definition with the header's fixed_part
static u128 general(df a, int frac) {
    uint64_t l1, h1, l2, h2;
    rs::fixed_part(a.hi, frac, l1, h1);
    rs::fixed_part(a.lo, frac, l2, h2);
    const uint64_t lo = l1 + l2;
    const uint64_t hi = h1 + h2 + (lo < l1 ? 1 : 0);
    if ((int64_t)hi < 0) return 0;
    return ((u128)hi << 64) | lo;
}

static long double val(df a) { return (long double)a.hi + (long double)a.lo; }
static long double rel(long double got, long double want) {
    return want == 0 ? fabsl(got) : fabsl(got - want) / fabsl(want);
}
// a positive double-float with a random 48-bit significand around 2^e
static df random_df(std::mt19937_64 &r, int e) {
    const float hi = std::ldexp(1.0f + (float)(r() >> 41) / 8388608.0f, e);
    const float lo = std::ldexp((float)(r() >> 41) / 8388608.0f - 0.5f, e - 24);
    return rs::quick_two_sum(hi, lo);
}

// the largest relative errors of the double-float operations, against long double
static int accuracy(long long cases) {
    std::mt19937_64 r(7);
    long double e_mul = 0, e_add = 0, e_div = 0, e_cbrt = 0;
    for (long long it = 0; it < cases; ++it) {
        const df a = random_df(r, (int)(r() % 40) - 20), b = random_df(r, (int)(r() % 40) - 20);
        e_mul = std::max(e_mul, rel(val(rs::df_mul(a, b)), val(a) * val(b)));
        e_add = std::max(e_add, rel(val(rs::df_add(a, b)), val(a) + val(b)));
        const uint32_t y = 1 + (uint32_t)(r() % 16777215u);
        e_div = std::max(e_div, rel(val(rs::df_div_u32(a, y)), val(a) / (long double)y));
        e_cbrt = std::max(e_cbrt, rel(val(rs::df_cbrt(a)), cbrtl(val(a))));
    }
    std::printf("max relative error: mul %.3Le add %.3Le div %.3Le cbrt %.3Le\n", e_mul, e_add, e_div, e_cbrt);
    const long double bound = 1.0L / (1LL << 44);
    return !(e_mul <= bound && e_add <= bound && e_div <= bound && e_cbrt <= bound);
}

int main(int argc, char **argv) {
    if (argc > 2 && std::strcmp(argv[1], "accuracy") == 0) return accuracy(atoll(argv[2]));
    const long long cases = argc > 1 ? atoll(argv[1]) : 10000000LL;
    std::mt19937_64 r(20261204);
    const int fracs[3] = {64, 58, 52};
    long long n = 0, bad = 0, shortpath = 0;
    for (long long it = 0; it < cases; ++it) {
        const uint32_t x = (uint32_t)r(), y = (uint32_t)r();
        float hi, lo;
        switch (it % 5) {
        case 0:                                      // arbitrary bit patterns, hi >= 0
            hi = __uint_as_float(x & 0x7FFFFFFFu);
            lo = __uint_as_float(y);
            break;
        case 1: case 2: {                            // normalised double-floats: |lo| <= ulp(hi) / 2
            const int e = 1 + (int)(x % 200);
            hi = __uint_as_float(((uint32_t)e << 23) | (y & 0x7FFFFFu));
            const int el = e - 24 - (int)(r() % 30);
            const uint32_t sgn = (uint32_t)(r() & 1) << 31;
            lo = el > 0 ? __uint_as_float(sgn | ((uint32_t)el << 23) | ((uint32_t)r() & 0x7FFFFFu)) : 0.0f;
            break;
        }
        case 3: {                                    // a trailing part too large for a normalised pair
            const int e = 60 + (int)(x % 100);
            hi = __uint_as_float(((uint32_t)e << 23) | (y & 0x7FFFFFu));
            const int el = e - (int)(r() % 26);
            lo = __uint_as_float(((uint32_t)(r() & 1) << 31) | ((uint32_t)el << 23) | ((uint32_t)r() & 0x7FFFFFu));
            break;
        }
        default:                                     // zeros, subnormals and products of double-floats
            if (x % 3 == 0) { hi = 0.0f; lo = 0.0f; }
            else if (x % 3 == 1) { hi = __uint_as_float(y & 0x7FFFFFu); lo = __uint_as_float(((uint32_t)r()) & 0x807FFFFFu); }
            else {
                const df a{std::ldexp((float)(y >> 8) / 16777216.0f + 0.5f, (int)(x % 20) - 10), 0.0f};
                const df b{std::ldexp((float)((uint32_t)r() >> 8) / 16777216.0f + 0.5f, (int)(r() % 20) - 10), 0.0f};
                const df p = rs::df_mul(rs::df_mul(a, b), rs::df_add(a, b));
                hi = p.hi; lo = p.lo;
            }
        }
        if (!std::isfinite(hi) || !std::isfinite(lo)) continue;
        const int frac = fracs[it % 3];
        const df a{hi, lo};
        const u128 got = rs::df_to_fixed(a, frac), want = general(a, frac);
        const int eh = (int)(__float_as_uint(hi) >> 23), el = (int)((__float_as_uint(lo) >> 23) & 0xFF);
        shortpath += ((unsigned)(eh - 150 + frac - 1) < 63u && el + 24 <= eh);
        ++n;
        if (got != want) {
            if (bad < 5) std::printf("mismatch hi=%a lo=%a frac=%d\n", hi, lo, frac);
            ++bad;
        }
    }
    std::printf("cases %lld short-path %lld mismatches %lld\n", n, shortpath, bad);
    return bad != 0 || shortpath == 0;
}
