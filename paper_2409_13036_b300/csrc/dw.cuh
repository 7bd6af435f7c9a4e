// Double-word ("float-float") arithmetic for the element and node passes.
//
// B300 issues FP64 operations, including float <-> double conversions, at 2 per clock per SM, against ~100 FP32
// FMAs per clock per SM, so a pass with a few dozen FP64 operations per element is bound by the FP64 pipe long
// before memory. A double-word value is an unevaluated sum h + l of two floats with |l| <= ulp(h) / 2: 48
// significant bits (unit roundoff u^2 = 2^-48 ~ 3.6e-15), computed on the FP32 pipes with error-free transforms:
//   two_sum (Knuth, TAOCP vol. 2, 4.2.2), fast_two_sum (Dekker 1971), two_prod via FMA;
//   add / add_fp / mul / mul_fp follow the double-word algorithms analysed by Joldes, Muller and Popescu,
//   "Tight and rigorous error bounds for basic building blocks of double-word arithmetic", ACM TOMS 44(2), 2017:
//   add = their accurate DW+DW (relative error < 3u^2), add_fast = the "sloppy" DW+DW (same-sign operands:
//   < 3u^2; otherwise an absolute error of a few u^2 (|x| + |y|)), add_fp = DW+FP (< 2u^2), mul = DW*DW with
//   three partial products (< 5u^2), mul_fp = DW*FP (< 2u^2).
// The intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn) keep the compiler from contracting or reordering the
// transforms. Conversions from and to double use integer operations only (see split / to_double), so that a
// pass reading and writing FP64 arrays issues one FP64 instruction per value written and none per value read.
#pragma once

#include <cuda_runtime.h>

namespace rafem {
namespace dw {

struct df {
    float h, l;
};

__device__ __forceinline__ df make(float h, float l = 0.0f) { return {h, l}; }

// s + e = a + b exactly, assuming |a| >= |b| or a == 0
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// s + e = a + b exactly, any a, b
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float ap = __fsub_rn(s, b);
    const float bp = __fsub_rn(s, ap);
    return {s, __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp))};
}

// p + e = a * b exactly (no underflow)
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df neg(df x) { return {-x.h, -x.l}; }

// x * 2^k for a power of two held as a float (exact barring under/overflow)
__device__ __forceinline__ df scale(df x, float pow2) { return {__fmul_rn(x.h, pow2), __fmul_rn(x.l, pow2)}; }

__device__ __forceinline__ df add(df x, df y) {
    const df s = two_sum(x.h, y.h);
    const df t = two_sum(x.l, y.l);
    const df v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}

__device__ __forceinline__ df add_fast(df x, df y) {
    const df s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}

__device__ __forceinline__ df sub(df x, df y) { return add(x, neg(y)); }

__device__ __forceinline__ df add_fp(df x, float y) {
    const df s = two_sum(x.h, y);
    return fast_two_sum(s.h, __fadd_rn(x.l, s.l));
}

__device__ __forceinline__ df mul(df x, df y) {
    const df c = two_prod(x.h, y.h);
    const float t0 = __fmul_rn(x.l, y.l);
    const float t1 = __fmaf_rn(x.h, y.l, t0);
    const float c2 = __fmaf_rn(x.l, y.h, t1);
    return fast_two_sum(c.h, __fadd_rn(c.l, c2));
}

__device__ __forceinline__ df mul_fp(df x, float y) {
    const df c = two_prod(x.h, y);
    return fast_two_sum(c.h, __fmaf_rn(x.l, y, c.l));
}

__device__ __forceinline__ df sqr(df x) {
    const df c = two_prod(x.h, x.h);
    const float t = __fmul_rn(__fadd_rn(x.h, x.h), x.l);
    return fast_two_sum(c.h, __fadd_rn(c.l, t));
}

// Compensated accumulation (Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6),
// 2005, algorithms Sum2 / Dot2): the running sum stays in y.h and the exact rounding errors of every product
// and addition, plus the cross terms of double-word operands, are gathered in y.l without renormalising, so an
// accumulated product costs 12 FP32 operations instead of the 20 of mul + add_fast. The result is as accurate
// as if computed in twice the precision and then rounded (an extra error of at most n^2 u^2 times the sum of
// the magnitudes for n terms). finish() renormalises with an exact two_sum.
__device__ __forceinline__ void dot_acc(df& y, df a, df b) {
    const df p = two_prod(a.h, b.h);
    const df s = two_sum(y.h, p.h);
    y.h = s.h;
    y.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, __fadd_rn(y.l, __fadd_rn(s.l, p.l))));
}

__device__ __forceinline__ void sum_acc(df& y, df a) {
    const df s = two_sum(y.h, a.h);
    y.h = s.h;
    y.l = __fadd_rn(y.l, __fadd_rn(s.l, a.l));
}

__device__ __forceinline__ df finish(df y) { return two_sum(y.h, y.l); }

// Double -> double-word with integer operations only. For a normal double with biased exponent e, h is x with
// its significand truncated to 24 bits (exactly representable as a float when 897 <= e <= 1150, i.e.
// 2^-126 <= |x| < 2^128) and the remainder x - h = r 2^(e-1075), r the 29 low significand bits, is rounded to a
// float by the integer-to-float conversion (an FP32-pipe instruction); a final fast_two_sum restores |l| <= ulp/2.
// 48 of the 53 significant bits survive. |x| < 2^-126 (zero included) gives 0; the callers' data (potentials,
// temperatures, conductances, volumes in SI units) stays far inside the range, which the context checks at create.
// |x| >= 2^128 gives an infinity of its sign (NaN stays NaN).
__device__ __forceinline__ df split(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu);
    const unsigned sign = hi & 0x80000000u;
    if (e < 897) return {0.0f, 0.0f};
    if (e > 1150) return {__uint_as_float(sign | 0x7f800000u | (e == 2047 && ((hi & 0xfffffu) | lo) ? 0x400000u : 0u)), 0.0f};
    const float h = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
    const float rm = __int2float_rn((int)(lo & 0x1fffffffu));
    float r;
    if (e >= 949) {
        r = __fmul_rn(rm, __uint_as_float((unsigned)(e - 948) << 23));  // 2^(e-1075)
    } else {
        // 2^(e-1075) is below the normal range: scale in two steps (the result may be subnormal)
        r = __fmul_rn(__fmul_rn(rm, __uint_as_float((unsigned)(e - 884) << 23)), __uint_as_float(63u << 23));
    }
    return fast_two_sum(h, __uint_as_float(__float_as_uint(r) | sign));
}

// float -> double of the same value with integer operations (normal floats, infinities and NaN; zero and
// subnormals give 0)
__device__ __forceinline__ double widen(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0) return 0.0;
    if (e == 255) return __hiloint2double((int)((b & 0x80000000u) | 0x7ff00000u | ((b & 0x7fffffu) ? 0x80000u : 0u)), 0);
    const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)((b & 7u) << 29));
}

// double-word -> nearest-ish double: one FP64 addition of the two exactly widened parts
__device__ __forceinline__ double to_double(df x) { return widen(x.h) + widen(x.l); }

// float2 storage of a double-word value (8 bytes, like the double it replaces)
__device__ __forceinline__ df load(const float2* p) {
    const float2 v = *p;
    return {v.x, v.y};
}
__device__ __forceinline__ df ldg(const float2* p) {
    const float2 v = __ldg(p);
    return {v.x, v.y};
}
__device__ __forceinline__ void store(float2* p, df x) { *p = make_float2(x.h, x.l); }

}  // namespace dw
}  // namespace rafem
