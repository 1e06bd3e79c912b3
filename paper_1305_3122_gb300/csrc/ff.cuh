// ff.cuh -- double-float ("ff") arithmetic on the FP32 pipes, with FP64 <-> ff conversions done by
// integer bit operations.
//
// GB300 runs FP32 fused multiply-adds about 58 times faster than FP64 ones, so the element
// arithmetic is carried out on unevaluated sums h + l of two floats (the double-word numbers of
// Dekker, "A floating-point technique for extending the available precision", Numer. Math. 18,
// 1971; error-free transforms as in Joldes, Muller, Popescu, "Tight and rigorous error bounds for
// basic building blocks of double-word arithmetic", ACM TOMS 44, 2017). Every operation below
// errs by a few units of 2^-48 relative to the magnitude of its operands (not of its result), so
// assembled values agree with FP64 to about 2^-45 of each row's largest entry.
//
// The conversions never touch the FP64 pipe:
//   ff_from_double  splits the 53-bit significand: hi keeps the top 24 bits (truncated), lo the
//                   next 29 bits rounded down to 24; |d - (hi + lo)| < 2^-47 |d|.
//   ff_to_double    builds the FP64 bit pattern of hi + lo directly (lo's bits below the 53-bit
//                   window are truncated, error < 2^-52 relative).
// Range: nonzero inputs need 2^-74 <= |d| < 2^128 (the lo part must stay a normal float);
// outside it `bad` is set and the value is treated as zero.
#pragma once

#include <stdint.h>

struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_make(float h) { return ff{h, 0.f}; }

__device__ __forceinline__ ff ff_from_double(double d, int& bad) {
    unsigned long long b = (unsigned long long)__double_as_longlong(d);
    unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
    unsigned sgn = hi32 & 0x80000000u;
    int e = (int)((hi32 >> 20) & 0x7FF) - 1023;
    if (e == -1023) {                                    // zero or subnormal
        if ((hi32 & 0xFFFFFu) | lo32) bad = 1;
        return ff{0.f, 0.f};
    }
    if (e > 127 || e < -74) {
        bad = 1;
        return ff{0.f, 0.f};
    }
    float h = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29));
    unsigned r = lo32 & 0x1FFFFFFFu;                      // remaining 29 bits, weight 2^(e-52)
    float l = 0.f;
    if (r) {
        int p = 31 - __clz(r);                           // leading bit, 0..28
        unsigned m = p >= 23 ? (r >> (p - 23)) : (r << (23 - p));
        int le = p + e - 52;                             // exponent of lo, >= -126 for e >= -74
        l = __uint_as_float(sgn | ((unsigned)(le + 127) << 23) | (m & 0x7FFFFFu));
    }
    return ff{h, l};
}

// The error-free transforms below must not be altered by the compiler's multiply-add
// contraction (fusing p + e with the product that made p, say, breaks their exactness), so each
// rounding step is written with the _rn intrinsics, which are never contracted; fmaf is used only
// where a fused operation is meant.
#define FADD(a, b) __fadd_rn((a), (b))
#define FSUB(a, b) __fsub_rn((a), (b))
#define FMUL(a, b) __fmul_rn((a), (b))

// s + t == a + b exactly (Knuth's two-sum), any magnitudes.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
    s = FADD(a, b);
    float bb = FSUB(s, a);
    t = FADD(FSUB(a, FSUB(s, bb)), FSUB(b, bb));
}

// h + l with |l| <= ulp(h)/2, from a possibly unnormalised pair.
__device__ __forceinline__ ff ff_norm(float h, float l) {
    float s, t;
    two_sum(h, l, s, t);
    return ff{s, t};
}

// s + t == a + b exactly when |a| >= |b| (fast two-sum).
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    float s = FADD(a, b);
    return ff{s, FSUB(b, FSUB(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = FADD(e, FADD(a.l, b.l));
    return ff_norm(s, e);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// Running sum acc += x, renormalised at every step so that each addition errs by at most a few
// units of 2^-48 of the running sum (carrying the low word unnormalised lets its own rounding
// grow with the number of terms).
__device__ __forceinline__ void ff_acc(ff& acc, ff x) { acc = ff_add(acc, x); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    float p = FMUL(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p, e);                          // |p| >= |e|
}

// ff times a float that is exact (a small integer or a power of two).
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
    float p = FMUL(a.h, b);
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    return fast_two_sum(p, e);
}

// a.x * b.x + a.y * b.y with one normalisation: error <= ~3 * 2^-48 (|ax bx| + |ay by|).
__device__ __forceinline__ ff ff_dot2(ff ax, ff ay, ff bx, ff by) {
    float p1 = FMUL(ax.h, bx.h);
    float e1 = fmaf(ax.h, bx.h, -p1);
    e1 = fmaf(ax.h, bx.l, e1);
    e1 = fmaf(ax.l, bx.h, e1);
    float p2 = FMUL(ay.h, by.h);
    float e2 = fmaf(ay.h, by.h, -p2);
    e2 = fmaf(ay.h, by.l, e2);
    e2 = fmaf(ay.l, by.h, e2);
    float s, e;
    two_sum(p1, p2, s, e);
    return ff_norm(s, FADD(e, FADD(e1, e2)));
}

// 1 / a: correctly rounded float reciprocal of the high part, then one Newton step in ff.
__device__ __forceinline__ ff ff_rcp(ff a) {
    float y = __frcp_rn(a.h);
    float r = fmaf(-a.h, y, 1.0f);
    r = fmaf(-a.l, y, r);
    return ff_norm(y, FMUL(y, r));
}

// FP64 value of h + l for a normalised pair (|l| <= ulp(h)/2, as every operation above returns),
// built bit by bit (no FP64 instruction).
__device__ __forceinline__ double ff_to_double(ff a) {
    float s = a.h, t = a.l;
    unsigned hb = __float_as_uint(s);
    int eh = (int)((hb >> 23) & 0xFF);
    if (eh == 0) return 0.0;                            // zero (float subnormals flush to zero)
    unsigned sg = hb >> 31;
    long long M = (long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;   // units of 2^(Eh - 52)
    unsigned lb = __float_as_uint(t);
    int el = (int)((lb >> 23) & 0xFF);
    if (el != 0) {
        long long Ml = (long long)((lb & 0x7FFFFFu) | 0x800000u);
        int sh = el - eh + 29;                          // <= 5 since |t| <= ulp(s)/2
        long long v = sh >= 0 ? (Ml << sh) : (sh > -40 ? (Ml >> -sh) : 0LL);
        M = ((lb >> 31) == sg) ? M + v : M - v;
    }
    int E = eh - 127;
    if (M >= (1LL << 53)) { M >>= 1; E += 1; }
    else if (M < (1LL << 52)) { M <<= 1; E -= 1; }
    unsigned long long bits = ((unsigned long long)sg << 63) | ((unsigned long long)(E + 1023) << 52) |
                              ((unsigned long long)M & ((1ULL << 52) - 1));
    return __longlong_as_double((long long)bits);
}
