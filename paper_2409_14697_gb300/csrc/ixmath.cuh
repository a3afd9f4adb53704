// Integer-product arithmetic ("IX") for complex128 gate updates.
//
// On GB300 the FP64 pipe issues 2 instructions per clock per SM, so a dense complex128
// one-qubit update (7-8 FP64 multiply-adds per amplitude, Eq. 2) runs at about a third
// of the HBM rate.  The integer pipes issue 64 (multiplies) to 128 (logic, shifts, adds)
// lanes per clock per SM.  This header evaluates each real output of an update,
//     y = sum_k c_k x_k      (c_k matrix entries with their signs, x_k amplitude parts),
// with integer instructions only, as a floating-point dot product with one wide
// accumulator and one final rounding:
//
//  * decode: a double x = +-M 2^(e - 1075), M in [2^52, 2^53), is kept as the 64-bit
//    significand M 2^11 (two 32-bit words, top bit set), its biased exponent e and its
//    sign (bit manipulation only; zero and subnormal inputs count as zero);
//  * products: the top 64 bits of the 128-bit product of two significands, from three
//    32x32-bit multiplies (the low x low word and the low halves of the cross words are
//    dropped: less than 3 units of the 64-bit result);
//  * alignment: the row's largest product exponent E is found first; every product is
//    shifted right by HEAD + (E - its exponent) bits, so the sum of up to 2^(HEAD-1)
//    terms fits a signed 64-bit accumulator whose unit is 2^(E + HEAD - 2108);
//  * result: the accumulator is rounded once to a double (round to nearest even) and
//    scaled by that unit, either with the integer-to-double conversion instruction
//    (I2F, an FP64-pipe instruction) or with integer instructions alone.  Both give the
//    same bits.
//
// Error: the accumulator carries at least 59 significant bits of the largest product
// (each term is off by less than 1.4 units, 4 terms by less than 5.5 units of 2^-59 of
// the largest |c_k x_k|), so every output is within 0.5 ulp of the exact sum plus
// 2^-56.4 max_k |c_k x_k|.  A chain of FP64 multiply-adds rounds after every term: its
// bound is about K ulp of the partial sums.  Limits: finite inputs; |x| below 2^-1022 is
// taken as 0; outputs whose unit falls below 2^-1022 (|y| < 2^-959) are flushed to 0;
// products must stay below 2^960.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define IX_HD __host__ __device__ __forceinline__
#else
#define IX_HD inline
#endif

namespace qs {
namespace ix {

// Exponent given to zero and subnormal inputs: its products shift out of every sum.
constexpr int32_t kZeroExp = -16384;

// A decoded double (or a matrix entry, decoded once on the host): significand (h:l) with
// bit 63 set, biased exponent e (kZeroExp for 0), sign mask s (0 or 0xFFFFFFFF).
struct Num {
    uint32_t h, l;
    int32_t e;
    uint32_t s;
};

IX_HD uint64_t bits_of(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
#endif
}

IX_HD double from_bits(uint64_t u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    std::memcpy(&x, &u, 8);
    return x;
#endif
}

// high 32 bits of (hi:lo) << s, 0 <= s < 32
IX_HD uint32_t funnel_l(uint32_t lo, uint32_t hi, int s) {
#ifdef __CUDA_ARCH__
    return __funnelshift_l(lo, hi, s);
#else
    return (uint32_t)((((uint64_t)hi << 32) | lo) << s >> 32);
#endif
}

IX_HD uint32_t umulhi(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// x >> s for any s (0 for s >= 64)
IX_HD uint64_t shr(uint64_t x, uint32_t s) {
#ifdef __CUDA_ARCH__
    uint64_t r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));  // PTX clamps s to 64
    return r;
#else
    return s >= 64 ? 0 : x >> s;
#endif
}

IX_HD Num decode(double x) {
    const uint64_t u = bits_of(x);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t e = (hi >> 20) & 0x7FFu;
    Num r;
    r.h = funnel_l(lo, hi, 11) | 0x80000000u;
    r.l = lo << 11;
    r.e = e ? (int32_t)e : kZeroExp;
    r.s = (uint32_t)((int32_t)hi >> 31);
    return r;
}

// floor(A B / 2^64) - d, 0 <= d < 3, for 64-bit significands A, B
IX_HD uint64_t mulhi(const Num &a, const Num &b) {
    return (uint64_t)a.h * b.h + umulhi(a.h, b.l) + umulhi(a.l, b.h);
}

// acc 2^k as a double, rounded to nearest even; k is the power of two of the
// accumulator's unit.  The conversion form uses the integer-to-double instruction.
IX_HD double encode_cvt(int64_t acc, int32_t k) {
#ifdef __CUDA_ARCH__
    const double d = __ll2double_rn(acc);
#else
    const double d = (double)acc;
#endif
    const uint64_t b = bits_of(d) + ((uint64_t)(int64_t)k << 52);
    return (acc == 0 || k < -1022) ? 0.0 : from_bits(b);
}

IX_HD int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

// The same with integer instructions only: |acc| normalised to bit 63, rounded at bit 10
// (from bit 62 after a one-bit shift, so the increment cannot carry out of 64 bits).
IX_HD double encode_int(int64_t acc, int32_t k) {
    const uint64_t sm = (uint64_t)(acc >> 63);
    const uint64_t mag = ((uint64_t)acc ^ sm) - sm;
    const int lz = clz64(mag);
    const uint64_t half = (mag << lz) >> 1;                      // bit 62 set
    const uint64_t m = (half + 0x1FFu + ((half >> 10) & 1u)) >> 10;  // [2^52, 2^53]
    // value = m 2^(52 - ... ): |acc| = half 2^(1 - lz), so |acc| 2^k = m 2^(11 - lz + k)
    const int64_t ef = (int64_t)(11 - lz + k) + 1075;  // biased exponent for m in [2^52, 2^53)
    const uint64_t b = ((uint64_t)(ef - 1) << 52) + m + (sm << 63);
    // k >= -1022 keeps ef >= 1 (lz <= 63); the conversion form flushes the same way
    return (mag == 0 || k < -1022) ? 0.0 : from_bits(b);
}

// One real output: sum over K terms of sign * c[k] * x[idx[k]], HEAD >= 1 + log2(K).
template <int K, int HEAD, bool CVT>
IX_HD double dot(const Num *x, const int (&idx)[K], const Num *c) {
    int32_t ep[K];
    int32_t E = kZeroExp * 2;
#pragma unroll
    for (int k = 0; k < K; k++) {
        ep[k] = x[idx[k]].e + c[k].e;
        E = ep[k] > E ? ep[k] : E;
    }
    int64_t acc = 0;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const Num &a = x[idx[k]];
        const uint64_t t = shr(mulhi(a, c[k]), (uint32_t)(E - ep[k]) + HEAD);
        const uint64_t sm = (uint64_t)(int64_t)(int32_t)(a.s ^ c[k].s);
        acc += (int64_t)((t ^ sm) - sm);
    }
    const int32_t k2 = E + HEAD - 2108;
    return CVT ? encode_cvt(acc, k2) : encode_int(acc, k2);
}

// A matrix entry with the sign its term takes (neg flips it).
IX_HD Num constant(double v, bool neg) {
    Num r = decode(v);
    if (neg) r.s = ~r.s;
    return r;
}

// ---- one-qubit updates (Eq. 2) ----------------------------------------------------
// ENC chooses each output's result encoding: 0 all by the conversion instruction, 2 all by
// integer instructions, 1 the real parts by conversion and the imaginary parts by integer
// instructions (the two give the same bits; the choice balances the FP64 and integer
// pipes).
constexpr bool enc_cvt(int enc, int out) { return enc == 0 || (enc == 1 && (out & 1) == 0); }

// Inputs x = (Re a, Im a, Re b, Im b) of an amplitude pair; outputs y in the same order,
// (a', b') = M (a, b) with M = [m00 m01; m10 m11] given as m[8] = m00r m00i m01r m01i
// m10r m10i m11r m11i.  Each row lists its terms' input indices; the host tables below
// give each term's matrix entry and sign.

// Term constants of the general 2x2 update (16) or, with r0 (Im m00 = 0: U3, CU3, RX,
// RY), of the 14-term form whose first two rows have 3 terms.
IX_HD void rows_dense1(Num *c, const double *m, bool r0) {
    int j = 0;
    if (r0) {
        c[j++] = constant(m[0], false); c[j++] = constant(m[2], false); c[j++] = constant(m[3], true);   // Re a': a.r b.r b.i
        c[j++] = constant(m[0], false); c[j++] = constant(m[2], false); c[j++] = constant(m[3], false);  // Im a': a.i b.i b.r
    } else {
        c[j++] = constant(m[0], false); c[j++] = constant(m[1], true);                  // Re a': a.r a.i
        c[j++] = constant(m[2], false); c[j++] = constant(m[3], true);                  //        b.r b.i
        c[j++] = constant(m[0], false); c[j++] = constant(m[1], false);                 // Im a': a.i a.r
        c[j++] = constant(m[2], false); c[j++] = constant(m[3], false);                 //        b.i b.r
    }
    c[j++] = constant(m[4], false); c[j++] = constant(m[5], true);                      // Re b': a.r a.i
    c[j++] = constant(m[6], false); c[j++] = constant(m[7], true);                      //        b.r b.i
    c[j++] = constant(m[4], false); c[j++] = constant(m[5], false);                     // Im b': a.i a.r
    c[j++] = constant(m[6], false); c[j++] = constant(m[7], false);                     //        b.i b.r
}

template <int ENC>
IX_HD void dense1_r0(const Num *c, const Num (&x)[4], double *y) {
    constexpr int r0[3] = {0, 2, 3}, i0[3] = {1, 3, 2}, r1[4] = {0, 1, 2, 3}, i1[4] = {1, 0, 3, 2};
    y[0] = dot<3, 3, enc_cvt(ENC, 0)>(x, r0, c + 0);
    y[1] = dot<3, 3, enc_cvt(ENC, 1)>(x, i0, c + 3);
    y[2] = dot<4, 3, enc_cvt(ENC, 2)>(x, r1, c + 6);
    y[3] = dot<4, 3, enc_cvt(ENC, 3)>(x, i1, c + 10);
}

template <int ENC>
IX_HD void dense1(const Num *c, const Num (&x)[4], double *y) {
    constexpr int r[4] = {0, 1, 2, 3}, i[4] = {1, 0, 3, 2};
    y[0] = dot<4, 3, enc_cvt(ENC, 0)>(x, r, c + 0);
    y[1] = dot<4, 3, enc_cvt(ENC, 1)>(x, i, c + 4);
    y[2] = dot<4, 3, enc_cvt(ENC, 2)>(x, r, c + 8);
    y[3] = dot<4, 3, enc_cvt(ENC, 3)>(x, i, c + 12);
}

// Real 2x2 (RY and other real rotations): 8 term constants, rows of 2 terms.
IX_HD void rows_dense1_real(Num *c, const double *m) {
    const double e[8] = {m[0], m[2], m[0], m[2], m[4], m[6], m[4], m[6]};
    for (int j = 0; j < 8; j++) c[j] = constant(e[j], false);
}

template <int ENC>
IX_HD void dense1_real(const Num *c, const Num (&x)[4], double *y) {
    constexpr int r[2] = {0, 2}, i[2] = {1, 3};
    y[0] = dot<2, 2, enc_cvt(ENC, 0)>(x, r, c + 0);
    y[1] = dot<2, 2, enc_cvt(ENC, 1)>(x, i, c + 2);
    y[2] = dot<2, 2, enc_cvt(ENC, 2)>(x, r, c + 4);
    y[3] = dot<2, 2, enc_cvt(ENC, 3)>(x, i, c + 6);
}

// Real diagonal, imaginary off-diagonal (RX): 8 term constants, rows of 2 terms.
IX_HD void rows_dense1_rx(Num *c, const double *m) {
    c[0] = constant(m[0], false); c[1] = constant(m[3], true);   // Re a': a.r b.i
    c[2] = constant(m[0], false); c[3] = constant(m[3], false);  // Im a': a.i b.r
    c[4] = constant(m[6], false); c[5] = constant(m[5], true);   // Re b': b.r a.i
    c[6] = constant(m[6], false); c[7] = constant(m[5], false);  // Im b': b.i a.r
}

template <int ENC>
IX_HD void dense1_rx(const Num *c, const Num (&x)[4], double *y) {
    constexpr int r0[2] = {0, 3}, i0[2] = {1, 2}, r1[2] = {2, 1}, i1[2] = {3, 0};
    y[0] = dot<2, 2, enc_cvt(ENC, 0)>(x, r0, c + 0);
    y[1] = dot<2, 2, enc_cvt(ENC, 1)>(x, i0, c + 2);
    y[2] = dot<2, 2, enc_cvt(ENC, 2)>(x, r1, c + 4);
    y[3] = dot<2, 2, enc_cvt(ENC, 3)>(x, i1, c + 6);
}

// Diagonal factors: element t times d[2t] + i d[2t+1]; 4 term constants per element.
IX_HD void rows_diag(Num *c, const double *d, int nt) {
    for (int t = 0; t < nt; t++) {
        c[4 * t + 0] = constant(d[2 * t], false);  // Re: x.r x.i
        c[4 * t + 1] = constant(d[2 * t + 1], true);
        c[4 * t + 2] = constant(d[2 * t], false);  // Im: x.i x.r
        c[4 * t + 3] = constant(d[2 * t + 1], false);
    }
}

// y = (dr + i di) x for a factor read per amplitude (diagonal tables): the factor is decoded
// on the spot.
template <int ENC>
IX_HD void cmul(double dr, double di, const Num (&x)[2], double *y) {
    const Num a = decode(dr), b = decode(di);
    Num c[4] = {a, b, a, b};
    c[1].s = ~c[1].s;
    constexpr int r[2] = {0, 1}, i[2] = {1, 0};
    y[0] = dot<2, 2, enc_cvt(ENC, 0)>(x, r, c + 0);
    y[1] = dot<2, 2, enc_cvt(ENC, 1)>(x, i, c + 2);
}

// x = (Re v, Im v) -> y = (Re, Im) of the product with one diagonal factor
template <int ENC>
IX_HD void phase(const Num *c, const Num (&x)[2], double *y) {
    constexpr int r[2] = {0, 1}, i[2] = {1, 0};
    y[0] = dot<2, 2, enc_cvt(ENC, 0)>(x, r, c + 0);
    y[1] = dot<2, 2, enc_cvt(ENC, 1)>(x, i, c + 2);
}

}  // namespace ix
}  // namespace qs
