// sem_dw.cuh -- double-word arithmetic: a value is a pair of FP32 numbers
// h + l (~48 significant bits), computed on the FP32 pipe with error-free
// transformations (Knuth's TwoSum; Dekker's product formed with one FMA) and
// FP32 low-order terms; and exact FP64 <-> double-word conversions in integer
// and FP32 arithmetic.  Used by the double-word operator (sem_ax_dw.cuh) and
// by the FP64 CG update's <r, r> reduction (sem_box.cuh).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace sem {

// A double-word number h + l.  Not normalised: l is the running sum of the
// low-order parts (the high part keeps the leading 24 bits; cancellation
// moves no error above 2^-48 of the operands' size).
struct alignas(8) dwf {
    float h, l;
};

// FP64 <-> double-word conversions in integer and FP32 arithmetic: GB300
// runs FP64 conversions on its FP64 pipe (1/64 rate), where a handful per
// node would cost as much as the double-word arithmetic itself.
//
// d -> (h, l): h = d rounded to 24 significant bits (half away from zero: a
// 2^28 carry into the 52-bit significand, then truncation), re-biased from
// the FP64 to the FP32 exponent; the remainder d - h is an exact signed
// 29-bit multiple m of d's last significand place 2^(e-1075); m is widened
// to FP32 exactly in two halves (float(k) = bits(2^23 + k) - 2^23, exact for
// |k| < 2^22) joined by one FMA (so l = rn(m) 2^(e-1075)), scaled by two
// powers of two (each representable for 2^-126 <= |d|), and given d's sign.
// |d| < 2^-126 (and zero) gives (+-0, 0); |d| >= 2^128 is outside the range.
__device__ __forceinline__ dwf dw_from_double(double d) {
    const uint64_t bits = uint64_t(__double_as_longlong(d));
    const uint32_t hi = uint32_t(bits >> 32);
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t e = (hi >> 20) & 0x7ffu;
    const uint64_t rb = bits + (uint64_t(1) << 28);
    const uint32_t hb = ((uint32_t(rb >> 29) - (384u << 23)) & 0x7fffffffu) | sign;
    const int32_t m = int32_t(uint32_t(rb) & 0x1fffffffu) - 0x10000000;
    const float fmh = __fsub_rn(__uint_as_float(0x4b400000u + uint32_t(m >> 14)), 12582912.0f);
    const float fml = __fsub_rn(__uint_as_float(0x4b000000u | (uint32_t(m) & 0x3fffu)), 8388608.0f);
    const float fm = __fmaf_rn(fmh, 16384.0f, fml);
    const float l = __fmul_rn(__fmul_rn(fm, 0x1p-52f), __uint_as_float((e - 896u) << 23));
    if (e < 897u) return {__uint_as_float(sign), 0.0f};
    return {__uint_as_float(hb), __uint_as_float(__float_as_uint(l) ^ sign)};
}

// Exact FP32 -> FP64 widening by re-biasing the exponent; zero and
// subnormal FP32 inputs (|f| < 2^-126) give a signed zero.
__device__ __forceinline__ double widen_f32(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t s = b & 0x80000000u;
    const bool normal = (b & 0x7f800000u) != 0u;
    const uint32_t hi = normal ? (s | (((b & 0x7fffffffu) >> 3) + (896u << 20))) : s;
    const uint32_t lo = normal ? (b << 29) : 0u;
    return __hiloint2double(int(hi), int(lo));
}

// h + l rounded once to FP64 (one FP64 addition).
__device__ __forceinline__ double dw_to_double(dwf v) { return widen_f32(v.h) + widen_f32(v.l); }

// s + e = a + b exactly (Knuth's TwoSum: no ordering of |a|, |b| needed).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

__device__ __forceinline__ dwf dw_add(dwf a, dwf b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    return {s, __fadd_rn(__fadd_rn(a.l, b.l), e)};
}

__device__ __forceinline__ dwf dw_sub(dwf a, dwf b) {
    float s, e;
    two_sum(a.h, -b.h, s, e);
    return {s, __fadd_rn(__fsub_rn(a.l, b.l), e)};
}

// c u: c.h u.h = p + e exactly (one FMA), the cross terms in FP32; c.l u.l
// (2^-48 of the product) is dropped.
__device__ __forceinline__ dwf dw_mul(dwf c, dwf u) {
    const float p = __fmul_rn(c.h, u.h);
    const float e = __fmaf_rn(c.h, u.h, -p);
    return {p, __fmaf_rn(c.l, u.h, __fmaf_rn(c.h, u.l, e))};
}

// acc + c u: the high product joins acc.h through TwoSum; every low-order
// term (product error, cross terms, sum error) goes to the low part.
__device__ __forceinline__ dwf dw_fma(dwf c, dwf u, dwf acc) {
    const float p = __fmul_rn(c.h, u.h);
    const float e = __fmaf_rn(c.h, u.h, -p);
    const float t = __fmaf_rn(c.l, u.h, __fmaf_rn(c.h, u.l, acc.l));
    float s, f;
    two_sum(acc.h, p, s, f);
    return {s, __fadd_rn(t, __fadd_rn(e, f))};
}

// acc + r^2 for an FP64 r: r = h + l exactly to ~2^-49, r^2 = h^2 + 2hl +
// l^2 with h^2 = p + e exactly (one FMA) and l^2 (2^-48 of r^2) dropped.
__device__ __forceinline__ dwf dw_add_square(dwf acc, double r) {
    const dwf v = dw_from_double(r);
    const float p = __fmul_rn(v.h, v.h);
    const float e = __fmaf_rn(v.h, v.h, -p);
    const float t = __fmaf_rn(__fmul_rn(2.0f, v.h), v.l, acc.l);
    float s, f;
    two_sum(acc.h, p, s, f);
    return {s, __fadd_rn(t, __fadd_rn(e, f))};
}

// acc + d r^2 for FP64 d, r (the Jacobi-weighted <r, M^-1 r> term):
// r^2 = p + (e + 2hl) as in dw_add_square, then times d's double-word form.
__device__ __forceinline__ dwf dw_add_weighted_square(dwf acc, double d, double r) {
    const dwf v = dw_from_double(r);
    const dwf w = dw_from_double(d);
    const float p = __fmul_rn(v.h, v.h);
    const float e = __fmaf_rn(v.h, v.h, -p);
    const dwf sq = {p, __fmaf_rn(__fmul_rn(2.0f, v.h), v.l, e)};
    return dw_fma(w, sq, acc);
}

}  // namespace sem
