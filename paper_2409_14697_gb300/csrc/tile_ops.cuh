// Applying a pass's ops to a tile held in shared memory (tile-local bit positions).
// Shared by the chunk kernel (K2) and the batched persistent kernel (K6).
#pragma once

#include <type_traits>

#include "dfmath.cuh"
#include "ixmath.cuh"
#include "kops.cuh"

namespace qs {


template <typename T>
__device__ __forceinline__ void ld_amp(const typename C2T<T>::type *p, Amp<T, 1> &a) {
    const auto v = *p;
    a.r[0] = v.x; a.i[0] = v.y;
}
template <typename T>
__device__ __forceinline__ void st_amp(typename C2T<T>::type *p, const Amp<T, 1> &a) {
    typename C2T<T>::type v;
    v.x = a.r[0]; v.y = a.i[0];
    *p = v;
}

template <typename T, int NT, typename Fn>
__device__ __forceinline__ void groups_apply(typename C2T<T>::type *tile, const KOp &op, int m, const Fn &fn) {
    const uint32_t ng = 1u << (m - op.nf);
    const uint32_t set = (uint32_t)op.set_mask;
    for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) {
        const uint32_t base = (uint32_t)insert_zero_bits(g, op.nf, op.fb) | set;
        Amp<T, 1> v[NT];
#pragma unroll
        for (int t = 0; t < NT; t++) ld_amp<T>(tile + (base + (uint32_t)op.off[t]), v[t]);
        fn(v);
#pragma unroll
        for (int t = 0; t < NT; t++) st_amp<T>(tile + (base + (uint32_t)op.off[t]), v[t]);
    }
}

// functors reading their matrix entries from shared memory (broadcast reads)
template <typename T> struct SH {
    T r;
    __device__ void operator()(Amp<T, 1> *v) const { f_h<T, 1>(v, r); }
};
// Unscaled Hadamard butterfly (a + b, a - b): 2 additions per amplitude.
template <typename T> struct SHSum {
    __device__ void operator()(Amp<T, 1> *v) const {
        const T ar = v[0].r[0], ai = v[0].i[0], br = v[1].r[0], bi = v[1].i[0];
        v[0].r[0] = ar + br; v[0].i[0] = ai + bi;
        v[1].r[0] = ar - br; v[1].i[0] = ai - bi;
    }
};
template <typename T> struct SSwap {
    __device__ void operator()(Amp<T, 1> *v) const { f_swap<T, 1>(v); }
};
template <typename T> struct SNeg {
    __device__ void operator()(Amp<T, 1> *v) const { f_neg<T, 1>(v); }
};
template <typename T> struct SDense1 {
    const T *m;
    __device__ void operator()(Amp<T, 1> *v) const { f_dense1<T, 1>(v, m); }
};
template <typename T> struct SDense1R0 {
    const T *m;
    __device__ void operator()(Amp<T, 1> *v) const { f_dense1_r0<T, 1>(v, m); }
};
template <typename T> struct SDense1Real {
    const T *m;
    __device__ void operator()(Amp<T, 1> *v) const { f_dense1_real<T, 1>(v, m); }
};
template <typename T> struct SDense1RX {
    const T *m;
    __device__ void operator()(Amp<T, 1> *v) const { f_dense1_rx<T, 1>(v, m); }
};
template <typename T> struct SDense2 {
    const T *m;
    __device__ void operator()(Amp<T, 1> *v) const { f_dense2<T, 1>(v, m); }
};
template <typename T, int NT> struct SDiag {
    const T *d;
    __device__ void operator()(Amp<T, 1> *v) const { f_diag<T, 1, NT>(v, d); }
};

// ---- complex128 integer-product forms (ixmath.cuh) of one-qubit dense and diagonal ops ----
// Each thread decodes the op's constants from the matrix reals in shared memory once; every
// fourth of its groups (iterations 0, 4, 8, ...) runs the native FP64 form, so the FP64 pipe
// and the integer pipes share the work, as in the streaming kernel.
constexpr uint32_t kIxNativeEvery = 4;

__device__ __forceinline__ void ix_load(const double2 &a, ix::Num (&x)[2]) {
    x[0] = ix::decode(a.x);
    x[1] = ix::decode(a.y);
}

template <int FORM>  // a D1_* class
__device__ __forceinline__ void ix_dense1_tile(double2 *tile, const KOp &op, int m, const double *sm) {
    ix::Num c[16];
    if (FORM == D1_R0) ix::rows_dense1(c, sm, true);
    else if (FORM == D1_REAL) ix::rows_dense1_real(c, sm);
    else if (FORM == D1_RX) ix::rows_dense1_rx(c, sm);
    else ix::rows_dense1(c, sm, false);
    const uint32_t ng = 1u << (m - op.nf);
    const uint32_t set = (uint32_t)op.set_mask;
    uint32_t it = 0;
    for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x, it++) {
        const uint32_t base = (uint32_t)insert_zero_bits(g, op.nf, op.fb) | set;
        double2 *pa = tile + (base + (uint32_t)op.off[0]);
        double2 *pb = tile + (base + (uint32_t)op.off[1]);
        const double2 a = *pa, b = *pb;
        double y[4];
        if (it % kIxNativeEvery == 0) {
            Amp<double, 1> v[2];
            v[0].r[0] = a.x; v[0].i[0] = a.y; v[1].r[0] = b.x; v[1].i[0] = b.y;
            if (FORM == D1_R0) f_dense1_r0<double, 1>(v, sm);
            else if (FORM == D1_REAL) f_dense1_real<double, 1>(v, sm);
            else if (FORM == D1_RX) f_dense1_rx<double, 1>(v, sm);
            else f_dense1<double, 1>(v, sm);
            y[0] = v[0].r[0]; y[1] = v[0].i[0]; y[2] = v[1].r[0]; y[3] = v[1].i[0];
        } else {
            const ix::Num x[4] = {ix::decode(a.x), ix::decode(a.y), ix::decode(b.x), ix::decode(b.y)};
            if (FORM == D1_R0) ix::dense1_r0<0>(c, x, y);
            else if (FORM == D1_REAL) ix::dense1_real<0>(c, x, y);
            else if (FORM == D1_RX) ix::dense1_rx<0>(c, x, y);
            else ix::dense1<0>(c, x, y);
        }
        *pa = make_double2(y[0], y[1]);
        *pb = make_double2(y[2], y[3]);
    }
}

// NT elements per group, element t times the factor (sm[2t], sm[2t+1])
template <int NT>
__device__ __forceinline__ void ix_diag_tile(double2 *tile, const KOp &op, int m, const double *sm) {
    ix::Num c[4 * NT];
    ix::rows_diag(c, sm, NT);
    const uint32_t ng = 1u << (m - op.nf);
    const uint32_t set = (uint32_t)op.set_mask;
    uint32_t it = 0;
    for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x, it++) {
        const uint32_t base = (uint32_t)insert_zero_bits(g, op.nf, op.fb) | set;
#pragma unroll
        for (int t = 0; t < NT; t++) {
            double2 *p = tile + (base + (uint32_t)op.off[t]);
            const double2 a = *p;
            double y[2];
            if (it % kIxNativeEvery == 0) {
                Amp<double, 1> v;
                v.r[0] = a.x; v.i[0] = a.y;
                f_diag<double, 1, 1>(&v, sm + 2 * t);
                y[0] = v.r[0]; y[1] = v.i[0];
            } else {
                ix::Num x[2];
                ix_load(a, x);
                ix::phase<0>(c + 4 * t, x, y);
            }
            *p = make_double2(y[0], y[1]);
        }
    }
}

template <typename T, int K>
__device__ __forceinline__ void dense_k_smem(typename C2T<T>::type *tile, const KOp &op, const T *m, int mbits) {
    constexpr int D = 1 << K;
    int sorted[K];
#pragma unroll
    for (int j = 0; j < K; j++) sorted[j] = op.pos[j];
#pragma unroll
    for (int a = 1; a < K; a++)
#pragma unroll
        for (int b = K - 1; b >= 1; b--)
            if (sorted[b - 1] > sorted[b]) {
                const int t = sorted[b]; sorted[b] = sorted[b - 1]; sorted[b - 1] = t;
            }
    uint32_t pbit[K];
#pragma unroll
    for (int j = 0; j < K; j++) pbit[j] = 1u << op.pos[j];
    auto offs = [&](int s) {
        uint32_t o = 0;
#pragma unroll
        for (int j = 0; j < K; j++) o |= ((s >> (K - 1 - j)) & 1) ? pbit[j] : 0u;
        return o;
    };
    const uint32_t ng = 1u << (mbits - K);
    for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) {
        uint32_t x = g;
#pragma unroll
        for (int j = 0; j < K; j++) {
            const int b = sorted[j];
            x = ((x >> b) << (b + 1)) | (x & ((1u << b) - 1u));
        }
        T vr[D], vi[D];
#pragma unroll
        for (int s = 0; s < D; s++) {
            Amp<T, 1> a;
            ld_amp<T>(tile + (x | offs(s)), a);
            vr[s] = a.r[0]; vi[s] = a.i[0];
        }
        // inputs are in registers, so each output row can be stored as soon as it is formed
#pragma unroll 1
        for (int r = 0; r < D; r++) {
            T ar = 0, ai = 0;
#pragma unroll
            for (int c = 0; c < D; c++) {
                const T mr = m[2 * (r * D + c)], mi = m[2 * (r * D + c) + 1];
                ar = fma(mr, vr[c], ar);
                ar = fma(-mi, vi[c], ar);
                ai = fma(mr, vi[c], ai);
                ai = fma(mi, vr[c], ai);
            }
            Amp<T, 1> a;
            a.r[0] = ar; a.i[0] = ai;
            st_amp<T>(tile + (x | offs(r)), a);
        }
    }
}

// ---- complex64 register phases (F_RPHASE) ---------------------------------------------
// A phase keeps the 2^kRpBits amplitudes spanned by kRpBits tile positions R (pos[0..4],
// register slot j <-> position pos[j]) in every thread's registers while a run of ops
// ("members") is applied to them, so the tile is read and written once per phase instead
// of once per op.  The other nt = m - kRpBits positions (off[0]: 4 bits each, ascending)
// are spelled by the thread index, bit i <-> i-th position; blockDim.x = 2^nt.
//
// Register r of lane l holds the amplitude whose R-bits are r ^ sigma(l).  sigma puts the
// positions 0..3 that lie in R on the upper lane bits of each half-warp, so the 16 lanes
// of an 8-byte shared-memory wavefront hit 16 different bank pairs whatever R is.  The
// members see the same operator in that register order: a 2x2 matrix on slot j is
// conjugated by X where bit j of sigma is set, and the bit masks of diagonals and controls
// are complemented on those slots.
//
// Program (floats, staged in shared memory): member count, then per member a code and
// `len` payload reals.  code = type | slot << 3 | a << 6 | b << 11 | len << 16, where a
// and b name positions: 16 + slot for a register position, the thread-index bit for any
// other, kRpAlways / kRpNever for a bit that is 1 / 0 for every amplitude.
//
// An exchange (X, or CNOT whose control is not a register position) is not carried out:
// it toggles bit `slot` of sigma, i.e. relabels which register holds which amplitude, and
// every later member and the final store read the relabelled order.
constexpr int kRpRegs = 1 << kRpBits;
static_assert(kRpMaxMembers * 9 + 1 <= kMaxOpReals, "a phase program must fit the staged reals");

// Bit r set iff bit j of r is set (j < kRpBits; index 5..7 unused).
static __constant__ uint32_t c_rp_pattern[8] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u, 0u, 0u, 0u};

__device__ __forceinline__ uint32_t rp_pattern(int j) { return c_rp_pattern[j & 7]; }

// The integer value of a float that holds one in [0, 2^23) (program codes and operand
// encodings): adding 2^23 puts it in the low mantissa bits, without a conversion
// instruction.
__device__ __forceinline__ uint32_t rp_int(float f) { return __float_as_uint(f + 8388608.0f) - 0x4B000000u; }

// Bit r of the result = the bit at operand position `enc` of the amplitude in register r.
// enc is the same for every thread of the block (it comes from the phase program).
__device__ __forceinline__ uint32_t rp_mask(int enc, uint32_t sigma, uint32_t tid) {
    if (enc == kRpAlways) return 0xFFFFFFFFu;
    if (enc == kRpNever) return 0u;
    if (enc & 16) {
        const int j = enc & 15;
        return rp_pattern(j) ^ (0u - ((sigma >> j) & 1u));
    }
    return 0u - ((tid >> enc) & 1u);
}

// True for an operand that names a register slot (its bit differs between registers).
__device__ __forceinline__ bool rp_is_slot(int enc) { return (enc & 16) && enc < kRpNever; }

// A mask that is the same for every register (an operand spelled by the thread index).
__device__ __forceinline__ bool rp_uniform(uint32_t K) { return K == 0u || K == 0xFFFFFFFFu; }

// Complex updates below are ordered so that every output's last multiply-add consumes the
// input it replaces (the other terms first, as partial sums): each result can then take
// its input's register, and the member loop needs no register copies.
__device__ __forceinline__ float2 rp_cmul(float2 a, float br, float bi) {
    const float pr = -a.y * bi, pi = a.x * bi;
    return make_float2(fmaf(a.x, br, pr), fmaf(a.y, br, pi));
}

// rows (M0 + i M1, M2 + i M3) and (M4 + i M5, M6 + i M7) applied to (x, y)
__device__ __forceinline__ void rp_2x2(const float (&M)[8], float2 &x, float2 &y) {
    float p0r = -M[1] * x.y;
    p0r = fmaf(M[2], y.x, p0r);
    p0r = fmaf(-M[3], y.y, p0r);
    float p0i = M[1] * x.x;
    p0i = fmaf(M[2], y.y, p0i);
    p0i = fmaf(M[3], y.x, p0i);
    float p1r = M[4] * x.x;
    p1r = fmaf(-M[5], x.y, p1r);
    p1r = fmaf(-M[7], y.y, p1r);
    float p1i = M[4] * x.y;
    p1i = fmaf(M[5], x.x, p1i);
    p1i = fmaf(M[7], y.x, p1i);
    x.x = fmaf(M[0], x.x, p0r);
    x.y = fmaf(M[0], x.y, p0i);
    y.x = fmaf(M[6], y.x, p1r);
    y.y = fmaf(M[6], y.y, p1i);
}

template <int J>
__device__ __forceinline__ void rp_m1(float2 (&v)[kRpRegs], const float (&M)[8]) {
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        if (r & (1 << J)) continue;
        rp_2x2(M, v[r], v[r | (1 << J)]);
    }
}

// real 2x2 (a b; c d): 4 multiply-adds per amplitude
template <int J>
__device__ __forceinline__ void rp_mr(float2 (&v)[kRpRegs], float a, float b, float c, float d) {
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        if (r & (1 << J)) continue;
        float2 &x = v[r], &y = v[r | (1 << J)];
        const float pxr = b * y.x, pxi = b * y.y, pyr = c * x.x, pyi = c * x.y;
        x.x = fmaf(a, x.x, pxr);
        x.y = fmaf(a, x.y, pxi);
        y.x = fmaf(d, y.x, pyr);
        y.y = fmaf(d, y.y, pyi);
    }
}

// (a, m01; m10, m11) with real a (U3 and one-qubit matrices like it): 7 multiply-adds per
// amplitude; P = a, m01 (re, im), m10 (re, im), m11 (re, im)
template <int J>
__device__ __forceinline__ void rp_mr0(float2 (&v)[kRpRegs], const float *P) {
    const float a = P[0], br = P[1], bi = P[2], cr = P[3], ci = P[4], dr = P[5], di = P[6];
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        if (r & (1 << J)) continue;
        float2 &x = v[r], &y = v[r | (1 << J)];
        float p0r = br * y.x;
        p0r = fmaf(-bi, y.y, p0r);
        float p0i = br * y.y;
        p0i = fmaf(bi, y.x, p0i);
        float p1r = cr * x.x;
        p1r = fmaf(-ci, x.y, p1r);
        p1r = fmaf(-di, y.y, p1r);
        float p1i = cr * x.y;
        p1i = fmaf(ci, x.x, p1i);
        p1i = fmaf(di, y.x, p1i);
        x.x = fmaf(a, x.x, p0r);
        x.y = fmaf(a, x.y, p0i);
        y.x = fmaf(dr, y.x, p1r);
        y.y = fmaf(dr, y.y, p1i);
    }
}

// (c0, i s01; i s10, c1) with real c0, s01, s10, c1 (RX): 4 multiply-adds per amplitude
template <int J>
__device__ __forceinline__ void rp_mx(float2 (&v)[kRpRegs], float c0, float s01, float s10, float c1) {
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        if (r & (1 << J)) continue;
        float2 &x = v[r], &y = v[r | (1 << J)];
        const float p1 = -s01 * y.y, p2 = s01 * y.x, p3 = -s10 * x.y, p4 = s10 * x.x;
        x.x = fmaf(c0, x.x, p1);
        x.y = fmaf(c0, x.y, p2);
        y.x = fmaf(c1, y.x, p3);
        y.y = fmaf(c1, y.y, p4);
    }
}

template <int J>
__device__ __forceinline__ void rp_c1(float2 (&v)[kRpRegs], const float (&M)[8], uint32_t K) {
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        if (r & (1 << J)) continue;
        float2 o0 = v[r], o1 = v[r | (1 << J)];
        rp_2x2(M, o0, o1);
        const bool c = (K >> r) & 1u;
        v[r] = c ? o0 : v[r];
        v[r | (1 << J)] = c ? o1 : v[r | (1 << J)];
    }
}

template <int J>
__device__ __forceinline__ void rp_x(float2 (&v)[kRpRegs], uint32_t K) {
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        if (r & (1 << J)) continue;
        const bool c = (K >> r) & 1u;
        const float2 x = v[r], y = v[r | (1 << J)];
        v[r] = c ? y : x;
        v[r | (1 << J)] = c ? x : y;
    }
}

__device__ __forceinline__ void rp_scale(float2 (&v)[kRpRegs], float dr, float di) {
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) v[r] = rp_cmul(v[r], dr, di);
}

__device__ __forceinline__ void rp_diag(float2 (&v)[kRpRegs], const float (&d)[8], uint32_t Ka, uint32_t Kb) {
    if (rp_uniform(Ka) && rp_uniform(Kb)) {
        const bool xa = Ka != 0u, xb = Kb != 0u;
        rp_scale(v, xa ? (xb ? d[6] : d[4]) : (xb ? d[2] : d[0]), xa ? (xb ? d[7] : d[5]) : (xb ? d[3] : d[1]));
        return;
    }
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        const bool xa = (Ka >> r) & 1u, xb = (Kb >> r) & 1u;
        const float dr = xa ? (xb ? d[6] : d[4]) : (xb ? d[2] : d[0]);
        const float di = xa ? (xb ? d[7] : d[5]) : (xb ? d[3] : d[1]);
        v[r] = rp_cmul(v[r], dr, di);
    }
}

// multiply by f where bit r of K is set, by e elsewhere
__device__ __forceinline__ void rp_two(float2 (&v)[kRpRegs], float er, float ei, float fr, float fi, uint32_t K) {
    if (rp_uniform(K)) {
        rp_scale(v, K ? fr : er, K ? fi : ei);
        return;
    }
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        const bool c = (K >> r) & 1u;
        v[r] = rp_cmul(v[r], c ? fr : er, c ? fi : ei);
    }
}

// negate where bit r of K is set (sign by multiplication: the FMA pipe, not the ALU)
__device__ __forceinline__ void rp_neg(float2 (&v)[kRpRegs], uint32_t K) {
    if (K == 0u) return;
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        const float s = __int_as_float(0x3f800000u | ((K << (31 - r)) & 0x80000000u));
        v[r].x *= s;
        v[r].y *= s;
    }
}

// multiply register r by table[c(r)] (re, im pairs), c(r) = the 4-bit count whose bit j is
// bit r of plane c_j.  The planes are first transposed into four words of nibbles (word i:
// nibble m is the count of register 4m + i), so a register's count costs a shift and a mask
// instead of four bit extracts.
__device__ __forceinline__ void rp_table(float2 (&v)[kRpRegs], const float *table, uint32_t c0, uint32_t c1,
                                         uint32_t c2, uint32_t c3) {
    if (rp_uniform(c0) && rp_uniform(c1) && rp_uniform(c2) && rp_uniform(c3)) {
        const int k = (int)((c0 & 1u) | (c1 & 2u) | (c2 & 4u) | (c3 & 8u));
        rp_scale(v, table[2 * k], table[2 * k + 1]);
        return;
    }
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; i++)
        w[i] = ((c0 >> i) & 0x11111111u) | (((c1 >> i) & 0x11111111u) << 1) | (((c2 >> i) & 0x11111111u) << 2) |
               (((c3 >> i) & 0x11111111u) << 3);
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        const uint32_t k2 = ((w[r & 3] >> (4 * (r >> 2))) & 15u) << 1;
        v[r] = rp_cmul(v[r], table[k2], table[k2 + 1]);
    }
}

__device__ __forceinline__ void rp_ph(float2 (&v)[kRpRegs], float pr, float pi, uint32_t K) {
    if (K == 0u) return;
    if (K == 0xFFFFFFFFu) {
        rp_scale(v, pr, pi);
        return;
    }
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        const float2 y = rp_cmul(v[r], pr, pi);
        v[r] = ((K >> r) & 1u) ? y : v[r];
    }
}

// Run form of RP_PH: multiply register r by T * prod_j (x_j(r) ? g_j : 1) * (-1)^(odd sign
// pairs), where T is the product of the phases on thread-index positions and g_j that of the
// phases on register slot j.  The slot factors are built as two tables over the register
// bits (slots 0-2: 8 entries, slots 3-4: 4) indexed by x = r ^ sigma, then permuted into
// register order by sigma's bits; each register then costs two complex multiplies.
__device__ __forceinline__ void rp_swap_if(bool c, float2 &a, float2 &b) {
    const float2 x = a, y = b;
    a = c ? y : x;
    b = c ? x : y;
}

__device__ __forceinline__ float2 rp_mul2(float2 a, float2 b) { return rp_cmul(a, b.x, b.y); }

__device__ __forceinline__ void rp_phase_run(float2 (&v)[kRpRegs], const float *P, int nf, int ns, uint32_t sigma,
                                             uint32_t tid) {
    float2 T = make_float2(1.f, 0.f), g0 = T, g1 = T, g2 = T, g3 = T, g4 = T;
    for (int q = 0; q < nf; q++) {
        const int enc = (int)rp_int(P[3 * q]);
        const float2 f = make_float2(P[3 * q + 1], P[3 * q + 2]);
        if (rp_is_slot(enc)) {
            switch (enc & 15) {
            case 0: g0 = rp_mul2(g0, f); break;
            case 1: g1 = rp_mul2(g1, f); break;
            case 2: g2 = rp_mul2(g2, f); break;
            case 3: g3 = rp_mul2(g3, f); break;
            default: g4 = rp_mul2(g4, f); break;
            }
        } else {
            const float2 t = rp_mul2(T, f);
            T = (rp_mask(enc, sigma, tid) & 1u) ? t : T;
        }
    }
    uint32_t K = 0;
    for (int q = 0; q < ns; q++) {
        const int e = (int)rp_int(P[3 * nf + q]);
        K ^= rp_mask(e & 31, sigma, tid) & rp_mask(e >> 5, sigma, tid);
    }
    float2 A[8], B[4];
    A[0] = T;
    A[1] = rp_mul2(T, g0);
    A[2] = rp_mul2(T, g1);
    A[3] = rp_mul2(A[1], g1);
#pragma unroll
    for (int i = 0; i < 4; i++) A[4 + i] = rp_mul2(A[i], g2);
    B[0] = make_float2(1.f, 0.f);
    B[1] = g3;
    B[2] = g4;
    B[3] = rp_mul2(g3, g4);
    // register r holds x = r ^ sigma: entry x of a table moves to register x ^ sigma
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const bool c = (sigma >> b) & 1u;
#pragma unroll
        for (int i = 0; i < 8; i++)
            if (!(i & (1 << b))) rp_swap_if(c, A[i], A[i | (1 << b)]);
    }
#pragma unroll
    for (int b = 0; b < 2; b++) {
        const bool c = (sigma >> (3 + b)) & 1u;
#pragma unroll
        for (int i = 0; i < 4; i++)
            if (!(i & (1 << b))) rp_swap_if(c, B[i], B[i | (1 << b)]);
    }
#pragma unroll
    for (int r = 0; r < kRpRegs; r++) {
        float2 d = rp_mul2(A[r & 7], B[r >> 3]);
        const uint32_t sgn = (K << (31 - r)) & 0x80000000u;
        d.x = __uint_as_float(__float_as_uint(d.x) ^ sgn);
        d.y = __uint_as_float(__float_as_uint(d.y) ^ sgn);
        v[r] = rp_mul2(v[r], d);
    }
}

// Tile index of register 0 of this thread (register r: base ^ XOR of pb[j] over the bits
// j of r), sigma and the per-slot position bits of phase ph.
__device__ __forceinline__ void rp_geometry(const KOp &ph, uint32_t tid, uint32_t (&pb)[kRpBits], uint32_t &base,
                                            uint32_t &sigma) {
    const uint32_t lane = tid & 31u;
    int nlow = 0;
#pragma unroll
    for (int j = 0; j < kRpBits; j++) {
        pb[j] = 1u << ph.pos[j];
        nlow += ph.pos[j] < 4 ? 1 : 0;
    }
    sigma = 0;
    int li = 4 - nlow;
#pragma unroll
    for (int j = 0; j < kRpBits; j++)
        if (ph.pos[j] < 4) {
            sigma |= ((lane >> li) & 1u) << j;
            li++;
        }
    base = 0;
    for (int i = 0; i < ph.nt; i++) base |= ((tid >> i) & 1u) << (uint32_t)((ph.off[0] >> (4 * i)) & 15u);
#pragma unroll
    for (int j = 0; j < kRpBits; j++) base ^= ((sigma >> j) & 1u) ? pb[j] : 0u;
}

template <int R>
__device__ __forceinline__ uint32_t rp_index(uint32_t base, const uint32_t (&pb)[kRpBits]) {
    uint32_t o = base;
#pragma unroll
    for (int j = 0; j < kRpBits; j++)
        if (R & (1 << j)) o ^= pb[j];
    return o;
}

template <int R>
__device__ __forceinline__ void rp_load(float2 (&v)[kRpRegs], const float2 *tile, uint32_t base,
                                        const uint32_t (&pb)[kRpBits]) {
    if constexpr (R < kRpRegs) {
        v[R] = tile[rp_index<R>(base, pb)];
        rp_load<R + 1>(v, tile, base, pb);
    }
}
template <int R>
__device__ __forceinline__ void rp_store(const float2 (&v)[kRpRegs], float2 *tile, uint32_t base,
                                         const uint32_t (&pb)[kRpBits]) {
    if constexpr (R < kRpRegs) {
        tile[rp_index<R>(base, pb)] = v[R];
        rp_store<R + 1>(v, tile, base, pb);
    }
}

// Runs one phase: every thread of the block must call this.
__device__ __forceinline__ void rphase_run(float2 *tile, const KOp &ph, const float *prog) {
    const uint32_t tid = threadIdx.x;
    float2 v[kRpRegs];
    uint32_t sigma;
    {
        uint32_t pb[kRpBits], base;
        rp_geometry(ph, tid, pb, base, sigma);
        rp_load<0>(v, tile, base, pb);
    }
    const int nmem = (int)rp_int(prog[0]);
    const float *mm = prog + 1;
    for (int i = 0; i < nmem; i++) {
        const int code = (int)rp_int(mm[0]);
        const int type = code & 7, J = (code >> 3) & 7, ea = (code >> 6) & 31, eb = (code >> 11) & 31;
        const int len = (code >> 16) & 255;
        const float *P = mm + 1;
        mm += 1 + len;
        switch (type) {
        case RP_M1:
            if (eb == RP_R0) {
                switch (J) {
                case 0: rp_mr0<0>(v, P); break;
                case 1: rp_mr0<1>(v, P); break;
                case 2: rp_mr0<2>(v, P); break;
                case 3: rp_mr0<3>(v, P); break;
                default: rp_mr0<4>(v, P); break;
                }
                break;
            }
            if (eb != RP_GENERAL) {
                // the 4-real forms: X M X reverses the payload order
                const int f = (int)((sigma >> J) & 1u);
                const float q0 = P[3 * f], q1 = P[1 + f], q2 = P[2 - f], q3 = P[3 - 3 * f];
                if (eb == RP_REAL) {
                    switch (J) {
                    case 0: rp_mr<0>(v, q0, q1, q2, q3); break;
                    case 1: rp_mr<1>(v, q0, q1, q2, q3); break;
                    case 2: rp_mr<2>(v, q0, q1, q2, q3); break;
                    case 3: rp_mr<3>(v, q0, q1, q2, q3); break;
                    default: rp_mr<4>(v, q0, q1, q2, q3); break;
                    }
                } else {
                    switch (J) {
                    case 0: rp_mx<0>(v, q0, q1, q2, q3); break;
                    case 1: rp_mx<1>(v, q0, q1, q2, q3); break;
                    case 2: rp_mx<2>(v, q0, q1, q2, q3); break;
                    case 3: rp_mx<3>(v, q0, q1, q2, q3); break;
                    default: rp_mx<4>(v, q0, q1, q2, q3); break;
                    }
                }
                break;
            }
            [[fallthrough]];
        case RP_C1: {
            // X M X in this lane's register order where bit J of sigma is set: the rows and
            // columns of the payload are read swapped
            const int f = (int)((sigma >> J) & 1u);
            float M[8];
            M[0] = P[6 * f]; M[1] = P[6 * f + 1];
            M[2] = P[2 + 2 * f]; M[3] = P[3 + 2 * f];
            M[4] = P[4 - 2 * f]; M[5] = P[5 - 2 * f];
            M[6] = P[6 - 6 * f]; M[7] = P[7 - 6 * f];
            if (type == RP_M1) {
                switch (J) {
                case 0: rp_m1<0>(v, M); break;
                case 1: rp_m1<1>(v, M); break;
                case 2: rp_m1<2>(v, M); break;
                case 3: rp_m1<3>(v, M); break;
                default: rp_m1<4>(v, M); break;
                }
            } else {
                const uint32_t K = rp_mask(ea, sigma, tid);
                switch (J) {
                case 0: rp_c1<0>(v, M, K); break;
                case 1: rp_c1<1>(v, M, K); break;
                case 2: rp_c1<2>(v, M, K); break;
                case 3: rp_c1<3>(v, M, K); break;
                default: rp_c1<4>(v, M, K); break;
                }
            }
            break;
        }
        case RP_X: {
            const uint32_t K = rp_mask(ea, sigma, tid);
            if (rp_uniform(K)) {  // the same for every register: relabel instead of moving
                sigma ^= (K & 1u) << J;
                break;
            }
            switch (J) {
            case 0: rp_x<0>(v, K); break;
            case 1: rp_x<1>(v, K); break;
            case 2: rp_x<2>(v, K); break;
            case 3: rp_x<3>(v, K); break;
            default: rp_x<4>(v, K); break;
            }
            break;
        }
        case RP_DIAG: {
            float M[8];
#pragma unroll
            for (int e = 0; e < 8; e++) M[e] = P[e];
            rp_diag(v, M, rp_mask(ea, sigma, tid), rp_mask(eb, sigma, tid));
            break;
        }
        case RP_NEG: {
            // J + 1 sign patterns x_a x_b, one (a | b << 5) per payload real: signs multiply
            uint32_t K = 0;
            for (int q = 0; q <= J; q++) {
                const int e = (int)rp_int(P[q]);
                K ^= rp_mask(e & 31, sigma, tid) & rp_mask(e >> 5, sigma, tid);
            }
            rp_neg(v, K);
            break;
        }
        case RP_PARITY:
            rp_two(v, P[0], P[1], P[2], P[3], rp_mask(ea, sigma, tid) ^ rp_mask(eb, sigma, tid));
            break;
        case RP_PARITYN: {
            // np parity patterns x_a xor x_b (one (a | b << 5) per payload real), then the
            // np + 1 factors for 0..np odd patterns: the odd count of every register is
            // kept in 4 bit planes (a ripple counter over the 32 registers at once)
            const int np = (len - 2) / 3;
            uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
            for (int q = 0; q < np; q++) {
                const int e = (int)rp_int(P[q]);
                const uint32_t M = rp_mask(e & 31, sigma, tid) ^ rp_mask(e >> 5, sigma, tid);
                uint32_t cy = c0 & M;
                c0 ^= M;
                uint32_t cz = c1 & cy;
                c1 ^= cy;
                cy = c2 & cz;
                c2 ^= cz;
                c3 ^= cy;
            }
            rp_table(v, P + np, c0, c1, c2, c3);
            break;
        }
        default:  // RP_PH: one phase, or a run of one-position phases and sign pairs
            if (J == 1) rp_phase_run(v, P, ea, eb, sigma, tid);
            else rp_ph(v, P[0], P[1], rp_mask(ea, sigma, tid) & rp_mask(eb, sigma, tid));
            break;
        }
    }
    // the addresses are rebuilt from shared memory rather than kept live through the
    // members; the register order is the final sigma (exchanges relabel it)
    asm volatile("" ::: "memory");
    {
        uint32_t pb[kRpBits], base, sg;
        rp_geometry(ph, tid, pb, base, sg);
#pragma unroll
        for (int j = 0; j < kRpBits; j++) base ^= (((sg ^ sigma) >> j) & 1u) ? pb[j] : 0u;
        rp_store<0>(v, tile, base, pb);
    }
}

// Applies one op to the tile; op and its matrix entries are in shared memory.  RP = false
// leaves the register-phase code out (kernels that never receive F_RPHASE ops keep their
// registers for themselves).
template <typename T, bool RP = true, bool IX = false>
__device__ __forceinline__ void apply_op_smem(typename C2T<T>::type *tile, const KOp &op, const T *sm, int m) {
    if constexpr (IX && std::is_same<T, double>::value) {
        // complex128 integer products (QS_PREC_IX64) for one-qubit dense ops and diagonal ops
        // with constant factors.  Diagonal blocks read from tables (F_DIAGK, F_CDIAGK,
        // F_HCDIAGK) stay native: decoding a factor per amplitude measured slower there.
        double2 *t2 = (double2 *)tile;
        switch (op.fkind) {
        case F_DENSE1:
            if (op.k == D1_REAL) ix_dense1_tile<D1_REAL>(t2, op, m, sm);
            else if (op.k == D1_RX) ix_dense1_tile<D1_RX>(t2, op, m, sm);
            else if (op.k == D1_R0) ix_dense1_tile<D1_R0>(t2, op, m, sm);
            else ix_dense1_tile<D1_GENERAL>(t2, op, m, sm);
            return;
        case F_DIAG1: ix_diag_tile<2>(t2, op, m, sm); return;
        case F_PHASE: ix_diag_tile<1>(t2, op, m, sm); return;
        case F_DIAG2: ix_diag_tile<4>(t2, op, m, sm); return;
        default:
            break;  // everything else in native FP64
        }
    }
    switch (op.fkind) {
    case F_H:  // scale in the reals when a pass defers it (1: the unscaled butterfly)
        if (op.nmat >= 1 && sm[0] == (T)1) groups_apply<T, 2>(tile, op, m, SHSum<T>{});
        else groups_apply<T, 2>(tile, op, m, SH<T>{op.nmat >= 1 ? sm[0] : (T)0.70710678118654752440});
        break;
    case F_SWAP: groups_apply<T, 2>(tile, op, m, SSwap<T>{}); break;
    case F_DENSE1:
        if constexpr (std::is_same<T, double>::value) {
            // complex128: the FP64 pipe is the limit, use the cheapest form
            if (op.k == D1_REAL) groups_apply<T, 2>(tile, op, m, SDense1Real<T>{sm});
            else if (op.k == D1_RX) groups_apply<T, 2>(tile, op, m, SDense1RX<T>{sm});
            else if (op.k == D1_R0) groups_apply<T, 2>(tile, op, m, SDense1R0<T>{sm});
            else groups_apply<T, 2>(tile, op, m, SDense1<T>{sm});
        } else {
            groups_apply<T, 2>(tile, op, m, SDense1<T>{sm});
        }
        break;
    case F_DIAG1: groups_apply<T, 2>(tile, op, m, SDiag<T, 2>{sm}); break;
    case F_PHASE: groups_apply<T, 1>(tile, op, m, SDiag<T, 1>{sm}); break;
    case F_NEG: groups_apply<T, 1>(tile, op, m, SNeg<T>{}); break;
    case F_DIAG2: groups_apply<T, 4>(tile, op, m, SDiag<T, 4>{sm}); break;
    case F_DENSE2: groups_apply<T, 4>(tile, op, m, SDense2<T>{sm}); break;
    case F_DIAGK: {
        const uint32_t N = 1u << m;
        for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
            uint32_t s = 0;
            for (int j = 0; j < op.k; j++) s |= ((x >> op.pos[j]) & 1u) << (op.k - 1 - j);
            Amp<T, 1> v;
            ld_amp<T>(tile + x, v);
            f_diag<T, 1, 1>(&v, sm + 2 * s);
            st_amp<T>(tile + x, v);
        }
        break;
    }
    case F_CDIAGK:
    case F_HCDIAGK: {
        const int kt = op.k, kc = op.nf;
        const uint32_t ng = 1u << (m - kc);
        // F_HCDIAGK (nf = 1): first the butterfly with the partner across the control bit
        const uint32_t hb = op.fkind == F_HCDIAGK ? 1u << op.pos[kt] : 0u;
        for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) {
            uint32_t x = g;
            for (int j = 0; j < kc; j++) {
                const int b = op.pos[kt + j];
                x = ((x >> b) << (b + 1)) | (x & ((1u << b) - 1u));
            }
            x |= (uint32_t)op.set_mask;
            uint32_t s = 0;
            for (int j = 0; j < kt; j++) s |= ((x >> op.pos[j]) & 1u) << (kt - 1 - j);
            Amp<T, 1> v;
            ld_amp<T>(tile + x, v);
            if (hb) {
                Amp<T, 1> u[2];
                ld_amp<T>(tile + (x ^ hb), u[0]);
                u[1] = v;
                SHSum<T>{}(u);
                st_amp<T>(tile + (x ^ hb), u[0]);
                v = u[1];
            }
            f_diag<T, 1, 1>(&v, sm + 2 * s);
            st_amp<T>(tile + x, v);
        }
        break;
    }
    case F_DENSEK:
        if (op.k == 3) dense_k_smem<T, 3>(tile, op, sm, m);
        else if (op.k == 4) dense_k_smem<T, 4>(tile, op, sm, m);
        break;
    case F_RPHASE:
        if constexpr (std::is_same<T, float>::value && RP) rphase_run(tile, op, sm);
        break;
    default:
        break;
    }
}

// ---- complex128 ops with double-float arithmetic (matrix reals as (hi, lo) pairs) --------
__device__ __forceinline__ df::F2 dfneg(df::F2 a) { return df::F2{-a.h, -a.l}; }

// ---- complex128 double-float tiles ------------------------------------------------------
// For a whole pass the tile holds every amplitude as four floats (re hi, re lo, im hi,
// im lo) in its own 16-byte slot: split once after the load and joined once before the
// store, so that the ops in between run on FP32 units only (the per-op join to double is
// an FP64 add per value, which bound the earlier double-float sweeps by the FP64 pipe).
// Values stay normalised pairs (|lo| <= ulp(hi) / 2) between ops.
struct DfAmp {
    df::F2 r, i;
};

__device__ __forceinline__ df::F2 df_norm(df::Acc a) {  // Fast2Sum of (s, c)
    const float h = __fadd_rn(a.s, a.c);
    return df::F2{h, __fsub_rn(a.c, __fsub_rn(h, a.s))};
}

__device__ __forceinline__ void df_tile_split(double2 *tile, int m) {
    for (uint32_t x = threadIdx.x; x < (1u << m); x += blockDim.x) {
        const double2 a = tile[x];
        const df::F2 r = df::split(a.x), i = df::split(a.y);
        reinterpret_cast<float4 *>(tile)[x] = make_float4(r.h, r.l, i.h, i.l);
    }
}
__device__ __forceinline__ void df_tile_join(double2 *tile, int m) {
    for (uint32_t x = threadIdx.x; x < (1u << m); x += blockDim.x) {
        const float4 f = reinterpret_cast<const float4 *>(tile)[x];
        tile[x] = make_double2(df::join(f.x, f.y), df::join(f.z, f.w));
    }
}

__device__ __forceinline__ DfAmp df_ld(const float4 *p) {
    const float4 f = *p;
    return DfAmp{df::F2{f.x, f.y}, df::F2{f.z, f.w}};
}
__device__ __forceinline__ void df_st(float4 *p, const DfAmp &a) { *p = make_float4(a.r.h, a.r.l, a.i.h, a.i.l); }

// a * d (complex, both as pairs), normalised
__device__ __forceinline__ DfAmp df_cmul(const DfAmp &a, df::F2 dr, df::F2 di) {
    df::Acc re = df::mul(dr, a.r);
    df::mac(re, dfneg(di), a.i);
    df::Acc im = df::mul(dr, a.i);
    df::mac(im, di, a.r);
    return DfAmp{df_norm(re), df_norm(im)};
}

template <int NT, typename Fn>
__device__ __forceinline__ void df_groups_apply(float4 *tile, const KOp &op, int m, const Fn &fn) {
    const uint32_t ng = 1u << (m - op.nf);
    const uint32_t set = (uint32_t)op.set_mask;
    for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) {
        const uint32_t base = (uint32_t)insert_zero_bits(g, op.nf, op.fb) | set;
        DfAmp v[NT];
#pragma unroll
        for (int t = 0; t < NT; t++) v[t] = df_ld(tile + (base + (uint32_t)op.off[t]));
        fn(v);
#pragma unroll
        for (int t = 0; t < NT; t++) df_st(tile + (base + (uint32_t)op.off[t]), v[t]);
    }
}

struct DtH {
    df::F2 r;
    __device__ void operator()(DfAmp *v) const {
        const DfAmp a = v[0], b = v[1];
        v[0].r = df_norm(df::scale(df::add(a.r, b.r), r));
        v[0].i = df_norm(df::scale(df::add(a.i, b.i), r));
        v[1].r = df_norm(df::scale(df::sub(a.r, b.r), r));
        v[1].i = df_norm(df::scale(df::sub(a.i, b.i), r));
    }
};
// Unscaled Hadamard butterfly (a + b, a - b) on double-float amplitudes.
struct DtHSum {
    __device__ void operator()(DfAmp *v) const {
        const DfAmp a = v[0], b = v[1];
        v[0].r = df_norm(df::add(a.r, b.r));
        v[0].i = df_norm(df::add(a.i, b.i));
        v[1].r = df_norm(df::sub(a.r, b.r));
        v[1].i = df_norm(df::sub(a.i, b.i));
    }
};
struct DtSwap {
    __device__ void operator()(DfAmp *v) const {
        const DfAmp t = v[0];
        v[0] = v[1];
        v[1] = t;
    }
};
struct DtNeg {
    __device__ void operator()(DfAmp *v) const {
        v[0].r = dfneg(v[0].r);
        v[0].i = dfneg(v[0].i);
    }
};
// y_r = sum_c m[r][c] x_c over NT touched elements (matrix as pairs, row-major re/im)
template <int NT> struct DtDense {
    const df::F2 *m;
    __device__ void operator()(DfAmp *v) const {
        DfAmp x[NT];
#pragma unroll
        for (int t = 0; t < NT; t++) x[t] = v[t];
#pragma unroll
        for (int r = 0; r < NT; r++) {
            const df::F2 *row = m + 2 * NT * r;
            df::Acc a = df::mul(row[0], x[0].r);
            df::Acc b = df::mul(row[0], x[0].i);
            df::mac(a, dfneg(row[1]), x[0].i);
            df::mac(b, row[1], x[0].r);
#pragma unroll
            for (int c = 1; c < NT; c++) {
                df::mac(a, row[2 * c], x[c].r);
                df::mac(a, dfneg(row[2 * c + 1]), x[c].i);
                df::mac(b, row[2 * c], x[c].i);
                df::mac(b, row[2 * c + 1], x[c].r);
            }
            v[r] = DfAmp{df_norm(a), df_norm(b)};
        }
    }
};
template <int NT> struct DtDiag {
    const df::F2 *d;
    __device__ void operator()(DfAmp *v) const {
#pragma unroll
        for (int t = 0; t < NT; t++) v[t] = df_cmul(v[t], d[2 * t], d[2 * t + 1]);
    }
};

// Applies one op to a double-float tile (df_tile_split done); sm holds the op's reals as
// (hi, lo) pairs.  Dense blocks of 3 or more qubits are applied in FP64 (the tile is
// joined, the op applied, and the tile split again); every thread of the block must call
// this.
__device__ __forceinline__ void apply_op_dftile(double2 *tile_raw, const KOp &op, const df::F2 *sm, double *sd,
                                                int m) {
    float4 *tile = reinterpret_cast<float4 *>(tile_raw);
    switch (op.fkind) {
    case F_H:  // scale in the reals when a pass defers it (1: the unscaled butterfly)
        if (op.nmat >= 1 && sm[0].h == 1.0f && sm[0].l == 0.0f) df_groups_apply<2>(tile, op, m, DtHSum{});
        else df_groups_apply<2>(tile, op, m, DtH{op.nmat >= 1 ? sm[0] : df::F2{0.70710677f, 1.21016175e-08f}});
        break;
    case F_SWAP: df_groups_apply<2>(tile, op, m, DtSwap{}); break;
    case F_NEG: df_groups_apply<1>(tile, op, m, DtNeg{}); break;
    case F_DENSE1: df_groups_apply<2>(tile, op, m, DtDense<2>{sm}); break;
    case F_DIAG1: df_groups_apply<2>(tile, op, m, DtDiag<2>{sm}); break;
    case F_PHASE: df_groups_apply<1>(tile, op, m, DtDiag<1>{sm}); break;
    case F_DIAG2: df_groups_apply<4>(tile, op, m, DtDiag<4>{sm}); break;
    case F_DENSE2: df_groups_apply<4>(tile, op, m, DtDense<4>{sm}); break;
    case F_DIAGK:
    case F_CDIAGK: {
        // table over the k positions pos[0..k-1]; F_CDIAGK visits only the elements with
        // its nf control positions pos[k..] (ascending) set
        const int kt = op.k, kc = op.fkind == F_CDIAGK ? op.nf : 0;
        const uint32_t ng = 1u << (m - kc);
        for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) {
            uint32_t x = g;
            for (int j = 0; j < kc; j++) {
                const int b = op.pos[kt + j];
                x = ((x >> b) << (b + 1)) | (x & ((1u << b) - 1u));
            }
            if (kc) x |= (uint32_t)op.set_mask;
            uint32_t s = 0;
            for (int j = 0; j < kt; j++) s |= ((x >> op.pos[j]) & 1u) << (kt - 1 - j);
            df_st(tile + x, df_cmul(df_ld(tile + x), sm[2 * s], sm[2 * s + 1]));
        }
        break;
    }
    default: {
        df_tile_join(tile_raw, m);
        for (int j = threadIdx.x; j < op.nmat; j += blockDim.x) sd[j] = (double)sm[j].h + (double)sm[j].l;
        __syncthreads();
        apply_op_smem<double>(tile_raw, op, sd, m);
        __syncthreads();
        df_tile_split(tile_raw, m);
        break;
    }
    }
}

}  // namespace qs
