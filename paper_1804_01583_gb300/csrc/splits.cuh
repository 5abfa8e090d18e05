// splits.cuh -- exact three-float splits of doubles and the compensated
// float-pair arithmetic built on them, for the FP64 sums that run on the FP32
// pipe: the sums of squares of the FP64 grid iteration and the dot products
// of the FP64 Arnoldi pass (on this GPU the FP64 pipe retires about 1/64 of
// the FP32 rate; each term keeps about 47 significant bits and the sums are
// compensated, as accurate as FP64 accumulation).
#pragma once

#include <stdint.h>

namespace kv {

// x 2^-sh = a1 + a2 + a3 exactly, from the bits of x: a1 carries the sign, the
// exponent and the leading 24 significant bits (mantissa bits 51..29), a2
// bits 28..6 and a3 bits 5..0, each an integer below 2^23 converted exactly
// (2^23 + m has m as its low mantissa bits) and scaled by powers of two.  sh is chosen
// by the host so that every |x| 2^-sh stays below 2^8; values whose scaled
// magnitude is below 2^-100 give zero: their squares lie more than 2^-180
// below the sums they enter, which are at least 2^-80 of the largest term
// wherever the iteration has not broken down.
struct F3 {
    float a1, a2, a3;
};

__device__ __forceinline__ float small_uint_to_float(unsigned m) {  // exact for m < 2^23
    return __fsub_rn(__uint_as_float(0x4B000000u | m), 8388608.0f);
}

__device__ __forceinline__ F3 split3(double x, int sh) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - sh;  // biased exponent of x 2^-sh
    F3 r;
    if (e < 1023 - 100) {
        r.a1 = r.a2 = r.a3 = 0.f;
        return r;
    }
    // 2^(e-1023) with the sign of x, as float bits (e - 1023 >= -100 > -127)
    const unsigned pbits = (hi & 0x80000000u) | ((unsigned)(e - 1023 + 127) << 23);
    const float P = __uint_as_float(pbits);
    // a1: the sign, the exponent and mantissa bits 51..29 (20 from hi, 3 from lo)
    r.a1 = __uint_as_float(pbits | (__funnelshift_l(lo, hi, 3) & 0x7fffffu));
    r.a2 = __fmul_rn(__fmul_rn(small_uint_to_float((lo >> 6) & 0x7fffffu), 0x1p-46f), P);
    r.a3 = __fmul_rn(__fmul_rn(small_uint_to_float(lo & 63u), 0x1p-52f), P);
    return r;
}

// x 2^-sh = a1 + a2 with a1 exact (the sign, the exponent and mantissa bits
// 51..29, as in split3) and a2 the remaining 29 bits rounded to a float
// (|a2 - rest| <= 2^-48 |x 2^-sh|): the two-part form for products, where
// 2^-48 is below what FP64 accumulation keeps anyway.  Same preconditions
// and flush as split3.
struct F2 {
    float a1, a2;
};
__device__ __forceinline__ F2 split2(double x, int sh) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - sh;
    F2 r;
    if (e < 1023 - 100) {
        r.a1 = r.a2 = 0.f;
        return r;
    }
    const unsigned sgn = hi & 0x80000000u;
    const unsigned pbits = sgn | ((unsigned)(e - 1023 + 127) << 23);
    r.a1 = __uint_as_float(pbits | (__funnelshift_l(lo, hi, 3) & 0x7fffffu));
    // bits 28..0 of the mantissa: (lo mod 2^29) 2^-29 in [0, 1), times 2^(e-1023-23)
    const float P23 = __uint_as_float(sgn | ((unsigned)(e - 1023 - 23 + 127) << 23));
    r.a2 = __fmul_rn(__fmul_rn(__uint2float_rn(lo & 0x1fffffffu), 0x1p-29f), P23);
    return r;
}

// a + b = s + e exactly (TwoSum, Knuth: six float operations, any magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Compensated float-pair accumulator of terms t = th + tl (hi + lo, the
// rounding errors of the additions kept in lo).
struct Acc2 {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float th, float tl) {
        float s, e;
        two_sum(hi, th, s, e);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(e, tl));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// square of x = a1 + a2 + a3 as a float pair: a1^2 exactly (TwoProduct), the
// cross terms 2 a1 (a2 + a3) and a2^2 in the low part (their rounding is
// 2^-48 of x^2)
__device__ __forceinline__ void sq3(const F3& x, float& th, float& tl) {
    th = __fmul_rn(x.a1, x.a1);
    const float e = __fmaf_rn(x.a1, x.a1, -th);
    const float a23 = __fadd_rn(x.a2, x.a3);
    tl = __fmaf_rn(__fadd_rn(x.a1, x.a1), a23, __fmaf_rn(x.a2, x.a2, e));
}

// (p - q)^2 as a float pair, p and q exact splits: the difference first as an
// unevaluated pair dh + dl accurate to about 2^-47 of |p - q| (the leading
// parts' difference and its error by TwoSum, the second parts' likewise),
// then squared as in sq3
__device__ __forceinline__ void sqdiff3(const F3& p, const F3& q, float& th, float& tl) {
    float s1, e1, s2, e2, u, f, dh, g;
    two_sum(p.a1, -q.a1, s1, e1);
    two_sum(p.a2, -q.a2, s2, e2);
    const float t3 = __fsub_rn(p.a3, q.a3);
    two_sum(s2, e1, u, f);
    two_sum(s1, u, dh, g);
    const float dl = __fadd_rn(g, __fadd_rn(__fadd_rn(f, e2), t3));
    th = __fmul_rn(dh, dh);
    const float e = __fmaf_rn(dh, dh, -th);
    tl = __fmaf_rn(__fadd_rn(dh, dh), dl, e);
}

}  // namespace kv
