// Double-float ("DF") arithmetic for complex128 gate updates on FP32 units.
//
// On GB300 the FP64 pipe issues 2 instructions per clock per SM, 1/64 of the FP32 rate,
// and FP64<->FP32 conversion instructions run on that same pipe.  A dense complex128
// one-qubit update needs 8 FP64 instructions per amplitude, which caps it far below the
// HBM rate.  This header evaluates the same update with FP32 arithmetic on value pairs:
//
//  * split: a double x is cut, with integer operations on its bit pattern, into
//    h = x truncated to 24 significant bits (exact) and l = the remainder x - h rounded to
//    24 bits (integer-to-float conversion of the 29 low mantissa bits, then an exact
//    power-of-two scale): x = h + l with |x - h - l| <= 2^-48 |x|;
//  * products: Dekker/Knuth TwoProd via FMA gives h_a*h_b exactly as (p, e); the cross
//    terms h_a*l_b + l_a*h_b are accumulated in FP32 (their rounding is ~2^-48 relative);
//  * sums of products: Knuth's TwoSum keeps the high parts' rounding errors exactly
//    (compensated dot product in the manner of Ogita, Rump and Oishi's Dot2);
//  * join: the pair (s, c) becomes double(s) + double(c) with one FP64 add; float->double
//    is rebuilt exactly from the float's bits with integer operations.
//
// Error: every output is within a few units of 2^-46 of sum |m_i x_i| of the exact
// value, far inside the 1e-12 amplitude tolerance for normalised states.  Values must be
// normal doubles below 2^127 in magnitude; magnitudes below 2^-100 are treated as 0
// (absolute error < 1e-30).
#pragma once

#include <cstdint>

namespace qs {
namespace df {

struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 split(double x) {
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t E = (hi >> 20) & 0x7FFu;
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t hb = sign | ((((hi & 0x7FFFFFFFu) - 0x38000000u) << 3) | (lo >> 29));
    const float scale = __uint_as_float((E - 948u) << 23);  // 2^(E - 1075)
    const float r = __fmul_rn(__uint2float_rn(lo & 0x1FFFFFFFu), scale);
    F2 o;
    // |x| < 2^-126: h is not a normal float, use 0; |x| < 2^-74: the remainder (< 2^-97)
    // is dropped (the scale would not be a normal float either)
    o.h = E >= 897u ? __uint_as_float(hb) : 0.0f;
    o.l = E >= 949u ? (sign ? -r : r) : 0.0f;
    return o;
}

// Exact float -> double from the bit pattern (zero and subnormal floats give 0).
__device__ __forceinline__ double widen(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t ef = (b >> 23) & 0xFFu;
    const uint32_t hi = (b & 0x80000000u) | (((b & 0x7FFFFFFFu) >> 3) + (896u << 20));
    const uint32_t lo = b << 29;
    return ef == 0 ? 0.0 : __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double join(float s, float c) { return __dadd_rn(widen(s), widen(c)); }

// Running compensated sum: value = s + c.
struct Acc {
    float s, c;
};

// acc := a * b (first term)
__device__ __forceinline__ Acc mul(F2 a, F2 b) {
    Acc r;
    r.s = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -r.s);
    e = fmaf(a.h, b.l, e);
    r.c = fmaf(a.l, b.h, e);
    return r;
}

// acc += a * b
__device__ __forceinline__ void mac(Acc &acc, F2 a, F2 b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    // TwoSum(acc.s, p)
    const float t = __fadd_rn(acc.s, p);
    const float bp = __fsub_rn(t, acc.s);
    const float err = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    acc.s = t;
    acc.c = __fadd_rn(acc.c, __fadd_rn(e, err));
}

// acc := a + b (pairs)
__device__ __forceinline__ Acc add(F2 a, F2 b) {
    Acc r;
    const float t = __fadd_rn(a.h, b.h);
    const float bp = __fsub_rn(t, a.h);
    const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(t, bp)), __fsub_rn(b.h, bp));
    r.s = t;
    r.c = __fadd_rn(err, __fadd_rn(a.l, b.l));
    return r;
}

// acc := a - b (pairs)
__device__ __forceinline__ Acc sub(F2 a, F2 b) {
    F2 nb;
    nb.h = -b.h;
    nb.l = -b.l;
    return add(a, nb);
}

// (s, c) * m, m a pair (the product of a compensated value and a constant)
__device__ __forceinline__ Acc scale(Acc v, F2 m) {
    Acc r;
    r.s = __fmul_rn(v.s, m.h);
    float e = fmaf(v.s, m.h, -r.s);
    e = fmaf(v.s, m.l, e);
    r.c = fmaf(v.c, m.h, e);
    return r;
}

__device__ __forceinline__ double result(Acc a) { return join(a.s, a.c); }

}  // namespace df
}  // namespace qs
