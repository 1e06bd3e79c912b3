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
// The conversions use the FP64 pipe at most once:
//   ff_from_double  splits the 53-bit significand: hi keeps the top 24 bits (truncated), lo the
//                   remaining 29 bits rounded to 24; |d - (hi + lo)| <= 2^-48 |d|.
//   ff_to_double    builds hi and lo as FP64 numbers bit by bit and adds them with one FP64
//                   addition (correctly rounded).
// Range: nonzero inputs need 2^-74 <= |d| < 2^128 (the lo part must stay a normal float);
// outside it `bad` is set and the value is treated as zero.
#pragma once

#include <stdint.h>

struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_make(float h) { return ff{h, 0.f}; }
__device__ __forceinline__ ff z_ff() { return ff{0.f, 0.f}; }

__device__ __forceinline__ ff ff_from_double(double d, int& bad) {
    unsigned hi32 = (unsigned)__double2hiint(d), lo32 = (unsigned)__double2loint(d);
    unsigned E = (hi32 >> 20) & 0x7FFu;                  // biased FP64 exponent, e = E - 1023
    unsigned sgn = hi32 & 0x80000000u;
    // hi: sign, float exponent e + 127 (= E - 896), the top 23 stored significand bits
    float h = __uint_as_float(__funnelshift_l(lo32, (hi32 & 0x7FFFFFFFu) - (896u << 20), 3) | sgn);
    // lo: the remaining 29 bits as an integer, rounded to a float and scaled by +-2^(e-52)
    float l = __uint2float_rn(lo32 & 0x1FFFFFFFu) * __uint_as_float(((E - 948u) << 23) | sgn);
    bool ok = E - 949u <= 201u;                          // -74 <= e <= 127
    if (!ok && E != 0u) bad = 1;                         // zero is exact; anything else out of range
    return ok ? ff{h, l} : ff{0.f, 0.f};
}

// The same for a computed value whose magnitude, when tiny, is a rounding residue: values below
// 2^-74 become zero without raising the range flag (only overflow does).
__device__ __forceinline__ ff ff_from_value(double d, int& bad) {
    unsigned E = ((unsigned)__double2hiint(d) >> 20) & 0x7FFu;
    if (E < 949u) return ff{0.f, 0.f};
    return ff_from_double(d, bad);
}

// Scaling by powers of two (exact): a group of FP64 inputs that enters a computation linearly
// (upstream gradients, say) is brought to magnitude about 1 by a common 2^k before the split,
// so that its range does not matter, and the results are scaled back by 2^-k in the conversion.
// Values below 2^-74 of the group's largest one become zero: they are negligible against it.

// k such that the largest |v| of the group times 2^k lies in [1, 2), from the biased FP64
// exponent emax of the largest value (0 for an all-zero group); clamped so that every
// conversion stays within the FP64 and float exponent ranges.
__device__ __forceinline__ int ff_group_scale(unsigned emax) {
    int k = emax ? 1023 - (int)emax : 0;
    return k < -100 ? -100 : (k > 800 ? 800 : k);
}

__device__ __forceinline__ unsigned fp64_biased_exponent(double d) { return ((unsigned)__double2hiint(d) >> 20) & 0x7FFu; }

// d * 2^k as a double-float (|d| 2^k <= 2^1 for the group's values).
__device__ __forceinline__ ff ff_from_double_scaled(double d, int k) {
    unsigned hi32 = (unsigned)__double2hiint(d), lo32 = (unsigned)__double2loint(d);
    int E = (int)((hi32 >> 20) & 0x7FFu);
    int Es = E + k;
    if (E == 0 || Es < 949 || Es > 1150) return ff{0.f, 0.f};
    unsigned sgn = hi32 & 0x80000000u;
    float h = __uint_as_float(sgn | ((unsigned)(Es - 896) << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29));
    float l = __uint2float_rn(lo32 & 0x1FFFFFFFu) * __uint_as_float(((unsigned)(Es - 948) << 23) | sgn);
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

// a + b: exact two-sum of the high words, low words added, one Fast2Sum to renormalise (the
// "sloppy" double-word sum of Joldes-Muller-Popescu). Error at most a few units of 2^-48 of
// |a| + |b| (not of |a + b|: cancellation is not compensated, and need not be here, because every
// sum's error is measured against the row's largest entry).
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = FADD(e, FADD(a.l, b.l));
    return fast_two_sum(s, e);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// Running sum acc += x, renormalised at every step so that each addition errs by at most a few
// units of 2^-48 of the running sum and the term (carrying the low word unnormalised lets its
// own rounding grow with the number of terms).
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

// a.x * b.x + a.y * b.y with one normalisation: error <= ~4 * 2^-48 (|ax bx| + |ay by|).
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
    return fast_two_sum(s, FADD(e, FADD(e1, e2)));
}

// |a|^2 = a.x^2 + a.y^2 (both terms non-negative: no cancellation, so the high words are summed
// with a Fast2Sum ordered by magnitude).
__device__ __forceinline__ ff ff_norm2(ff ax, ff ay) {
    float p1 = FMUL(ax.h, ax.h);
    float e1 = fmaf(ax.h, ax.h, -p1);
    e1 = fmaf(FADD(ax.h, ax.h), ax.l, e1);
    float p2 = FMUL(ay.h, ay.h);
    float e2 = fmaf(ay.h, ay.h, -p2);
    e2 = fmaf(FADD(ay.h, ay.h), ay.l, e2);
    ff s = fast_two_sum(fmaxf(p1, p2), fminf(p1, p2));
    return fast_two_sum(s.h, FADD(s.l, FADD(e1, e2)));
}

// 1 / a: correctly rounded float reciprocal of the high part, then one Newton step in ff.
__device__ __forceinline__ ff ff_rcp(ff a) {
    float y = __frcp_rn(a.h);
    float r = fmaf(-a.h, y, 1.0f);
    r = fmaf(-a.l, y, r);
    return fast_two_sum(y, FMUL(y, r));
}

// 1/a from the approximate float reciprocal and one Newton step in double-float (about 46 bits).
__device__ __forceinline__ ff ff_rcp_fast(ff a) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.h));
    float r = fmaf(-a.h, y, 1.0f);
    r = fmaf(-a.l, y, r);
    return fast_two_sum(y, FMUL(y, r));
}

// FP64 value of a float, built bit by bit (no conversion instruction): sign, exponent rebiased
// from 127 to 1023, significand shifted into place. Zero (and flushed subnormals) give 0.
__device__ __forceinline__ double f2d_bits(float f) {
    unsigned b = __float_as_uint(f);
    unsigned hi = (((b & 0x7FFFFFFFu) >> 3) + (896u << 20)) | (b & 0x80000000u);
    hi = (b & 0x7F800000u) ? hi : 0u;
    return __hiloint2double((int)hi, (int)(b << 29));
}

// FP64 value of h + l: both words are exact in FP64, so one FP64 addition gives h + l correctly
// rounded (the only FP64 instruction of the conversion).
__device__ __forceinline__ double ff_to_double(ff a) { return f2d_bits(a.h) + f2d_bits(a.l); }

// f * 2^-k as FP64, built bit by bit (k as from ff_group_scale, so the result stays normal).
__device__ __forceinline__ double f2d_bits_scaled(float f, int k) {
    unsigned b = __float_as_uint(f);
    unsigned hi = (((b & 0x7FFFFFFFu) >> 3) + ((unsigned)(896 - k) << 20)) | (b & 0x80000000u);
    hi = (b & 0x7F800000u) ? hi : 0u;
    return __hiloint2double((int)hi, (int)(b << 29));
}

// (h + l) * 2^-k as FP64 (one FP64 addition).
__device__ __forceinline__ double ff_to_double_scaled(ff a, int k) { return f2d_bits_scaled(a.h, k) + f2d_bits_scaled(a.l, k); }
