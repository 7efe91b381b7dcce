// rs_device.cuh -- device helpers shared by the scoring kernels and the
// incremental (serving) kernels.  Both must evaluate every term with the same
// operations in the same order, so that a score updated by deltas equals,
// bit for bit, the score recomputed from scratch.
#pragma once
#include "rs_internal.cuh"

namespace rs {

#ifndef RS_FULL_MASK
#define RS_FULL_MASK 0xFFFFFFFFu
#endif

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t dev_pow2_at_least(uint32_t x) {
    return x <= 1 ? 1u : 1u << (32 - __clz(x - 1));
}

__device__ __forceinline__ unsigned long long double_bits(df a) {
    return (unsigned long long)__double_as_longlong(df_to_double(a));
}

// ---- hash tables keyed by community (shared or global memory) ----------------
struct Tab {
    int32_t *key;
    uint32_t *cnt;
    unsigned long long *q;   // 2 words per slot (Type-II sums), may be null
    df *sig;                 // per slot sigma, may be null
    uint32_t mask;
};

__device__ __forceinline__ uint32_t slot_of(int32_t c, uint32_t mask) {
    uint32_t h = hash_label(c);
    h ^= h >> 15;
    return h & mask;
}

__device__ __forceinline__ int tab_insert(const Tab &t, int32_t c, uint32_t add, int *err) {
    uint32_t h = slot_of(c, t.mask);
    for (uint32_t it = 0; it <= t.mask; ++it) {
        int32_t prev = atomicCAS(&t.key[h], kEmpty, c);
        if (prev == kEmpty || prev == c) {
            if (add) atomicAdd(&t.cnt[h], add);
            return (int)h;
        }
        h = (h + 1) & t.mask;
    }
    atomicOr(err, 1);
    return -1;
}

// insert, returning the count before the add and whether the key is new
__device__ __forceinline__ int tab_insert_old(const Tab &t, int32_t c, uint32_t add, uint32_t &old, bool &fresh,
                                              int *err) {
    uint32_t h = slot_of(c, t.mask);
    for (uint32_t it = 0; it <= t.mask; ++it) {
        int32_t prev = atomicCAS(&t.key[h], kEmpty, c);
        if (prev == kEmpty || prev == c) {
            fresh = prev == kEmpty;
            old = atomicAdd(&t.cnt[h], add);
            return (int)h;
        }
        h = (h + 1) & t.mask;
    }
    atomicOr(err, 1);
    old = 0;
    fresh = false;
    return -1;
}

__device__ __forceinline__ int tab_find(const Tab &t, int32_t c) {
    uint32_t h = slot_of(c, t.mask);
    for (uint32_t it = 0; it <= t.mask; ++it) {
        int32_t k = t.key[h];
        if (k == c) return (int)h;
        if (k == kEmpty) return -1;
        h = (h + 1) & t.mask;
    }
    return -1;
}

// Type-II term sigma^2 (Q - s_u) in accumulator units (0 when rest or sigma is 0)
__device__ __forceinline__ u128 type2_term(df sig, u128 rest) {
    if (rest == 0 || !(sig.hi > 0.0f)) return 0;
    df t = df_mul(df_mul(sig, sig), df_from_u128(rest, -kSFrac));
    return df_to_fixed(t, kAccFrac);
}
// pushed to u (taken away, modulo 2^128, when neg)
__device__ __forceinline__ void push_type2(unsigned long long *acc, int32_t u, df sig, u128 rest, bool neg = false) {
    u128 v = type2_term(sig, rest);
    if (v) atomic_add_u128(acc + 2 * (int64_t)u, neg ? (u128)0 - v : v);
}

// The strict reading of the triad indicator (RS_TRIAD_STRICT) drops the closed
// triads (u, w, v) with C(v) = C(u) != C(w) and v in N(u): the Type-II sum
// Q_w(C(u)) - s_u pushed by w to u then leaves out X(w, u), the s of u's
// same-community neighbours that are also neighbours of w.  X is summed exactly
// per pushed pair beforehand, two words per CSR entry, at u's entry in w's row
// (sx null: the default reading).
struct Strict {
    const int32_t *col;
    const unsigned long long *sx;
};
__device__ __forceinline__ u128 strict_rest(const Strict &SX, const int64_t *off, int32_t w, int32_t u, u128 rest,
                                            int64_t pos = -1) {
    if (!SX.sx || rest == 0) return rest;
    if (pos < 0) {
        int64_t lo = off[w], hi = off[w + 1];
        while (lo < hi) {
            int64_t mid = lo + ((hi - lo) >> 1);
            if (SX.col[mid] < u) lo = mid + 1; else hi = mid;
        }
        pos = lo;
    }
    return rest - (((u128)SX.sx[2 * pos + 1] << 64) | SX.sx[2 * pos]);
}

// the three apex terms of triangle (a, b, c) from its six directed values
// S(x -> y) = w_x(C(y))^(1/3): at apex a the ordered pairs (w, v) = (b, c) and
// (c, b) give S(c->a) S(b->c) S(b->a) + S(b->a) S(c->b) S(c->a)
struct TriTerms { u128 a, b, c; };
// the same with the pair sums Pac = S(a->c) + S(c->a) and Pab = S(a->b) + S(b->a)
// given (df_add(Sac, Sca) and df_add(Sab, Sba)): the same operations, so the same bits
__device__ __forceinline__ TriTerms triangle_term_values_p(df Sab, df Sba, df Sac, df Sca, df Sbc, df Scb, df Pac,
                                                           df Pab) {
    df ta = df_mul(df_mul(Sba, Sca), df_add(Sbc, Scb));
    df tb = df_mul(df_mul(Sab, Scb), Pac);
    df tc = df_mul(df_mul(Sac, Sbc), Pab);
    return TriTerms{df_to_fixed(ta, kAccFrac), df_to_fixed(tb, kAccFrac), df_to_fixed(tc, kAccFrac)};
}
__device__ __forceinline__ TriTerms triangle_term_values(df Sab, df Sba, df Sac, df Sca, df Sbc, df Scb) {
    return triangle_term_values_p(Sab, Sba, Sac, Sca, Sbc, Scb, df_add(Sac, Sca), df_add(Sab, Sba));
}
__device__ __forceinline__ void add_triangle(unsigned long long *acc, int32_t a, int32_t b, int32_t c,
                                             const TriTerms &t, bool neg = false) {
    atomic_add_u128(acc + 2 * (int64_t)a, neg ? (u128)0 - t.a : t.a);
    atomic_add_u128(acc + 2 * (int64_t)b, neg ? (u128)0 - t.b : t.b);
    atomic_add_u128(acc + 2 * (int64_t)c, neg ? (u128)0 - t.c : t.c);
}

// finishing a row in P1: the row's largest weight, s_v and the node record;
// w_own is the weight of the row's own community when own > 0 (else ignored)
__device__ __forceinline__ df p1_row_result(const RowAgg &a, uint32_t own, df col_max, int32_t k,
                                            const uint64_t *LG, NodeRec &out, int32_t cv, df w_own,
                                            bool want_max) {
    df m = col_max;
    df wabs{0.0f, 0.0f};
    bool absent_col = want_max && a.L < (uint32_t)k;
    if (absent_col || own == 0) wabs = column_weight(a, 0, LG);   // community absent from N(v)
    if (absent_col) m = df_max(m, wabs);
    df wown = own > 0 ? w_own : wabs;
    df s = df_cbrt(wown);
    out.s_fix = (uint64_t)df_to_fixed(s, kSFrac);
    out.label = cv;
    out.dx = (int32_t)(a.T - own);
    return m;
}

}  // namespace rs
