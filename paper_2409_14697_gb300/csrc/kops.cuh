// Kernel-side form of one operation ("KOp") and the functors that apply it to the
// touched amplitudes of one group.  Shared by the streaming kernel (K1, groups over the
// whole state in HBM) and the chunk kernel (K2, groups over a tile in shared memory).
//
// Group structure (Eq. 2 / Eq. 3 of QueenV2, generalised): every group is one base index
// with the nf fixed bits fb[] cleared and the set_mask bits forced to one; the op reads
// and writes the nt elements at base | off[t].  Structure-specific kinds avoid touching
// amplitudes a gate leaves unchanged (controls, phases) and avoid arithmetic for
// permutations.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace qs {

enum FKind : int32_t {
    F_H = 0,     // (a+b, a-b)/sqrt2, nt = 2
    F_SWAP,      // exchange two elements, nt = 2
    F_DENSE1,    // 2x2 matrix, nt = 2 (m: 8 reals)
    F_DIAG1,     // diag(d0, d1), nt = 2 (m: 4 reals)
    F_PHASE,     // one element times e^{i a}, nt = 1 (m: 2 reals)
    F_NEG,       // one element times -1, nt = 1
    F_DIAG2,     // four phases, nt = 4 (m: 8 reals)
    F_DENSE2,    // 4x4 matrix, nt = 4 (m: 32 reals)
    F_DIAGK,     // diagonal on k qubits at positions pos[] (m: 2^(k+1) reals), every element
    F_DENSEK,    // dense 2^k x 2^k on positions pos[] (m: 2^(2k+1) reals), k = 3..6
    F_TC,        // dense block on the tensor cores (k = 4..6; mat/nmat index the B operand)
    F_RPHASE,    // complex64 register phase: a run of ops on 2^5 amplitudes per thread in registers
    F_CDIAGK,    // tile passes: diagonal over k table positions pos[0..k-1] on the elements whose
                 // nf control positions pos[k..k+nf-1] (ascending, set_mask) are all set; nt
                 // terms after the table, (table bit or -1, global qubit h, re, im): where
                 // bit h of the tile is 1, entries with that table bit set (all for -1) take
                 // the factor (the kernel folds them into a per-tile copy of the table);
                 // off[0] bit tb + 1 marks the table bits that have terms
    F_HCDIAGK,   // tile passes, complex128 FP64: the unscaled Hadamard butterfly (a + b, a - b)
                 // on the single control pos[k] of an F_CDIAGK, then that F_CDIAGK (fields
                 // as there, nf = 1): one sweep instead of two
};

// Structure of an F_DENSE1 matrix (FP64 operations per amplitude for complex128 work):
// general 8, real first entry 7 (U3, CU3), real 4 (RY), real diagonal with imaginary
// off-diagonal 4 (RX).
enum D1Class : int32_t { D1_GENERAL = 0, D1_R0 = 1, D1_REAL = 2, D1_RX = 3 };

// Reals staged in shared memory per op (dense 4-qubit block: 2 * 16 * 16).
constexpr int kMaxOpReals = 512;
// Threads per CTA of the tile kernels (chunk pass, batched launch).
constexpr int kTileThreadBits = 8;
constexpr int kTileThreads = 1 << kTileThreadBits;

// Register phases (F_RPHASE, complex64): kRpBits tile positions per thread in registers,
// so tiles of 2^(kTileThreadBits + kRpBits) amplitudes.  Member types of a phase program:
constexpr int kRpBits = 5;
constexpr int kRpAlways = 31;     // position operand whose bit is 1 for every amplitude
constexpr int kRpNever = 30;      // position operand whose bit is 0 for every amplitude
constexpr int kRpMaxMembers = 56; // ops per phase: 1 + 9 * 56 reals <= kMaxOpReals
enum RpType : int {
    RP_M1 = 0,  // 2x2 matrix on register slot `slot`; operand b holds its form: RP_GENERAL
                // (8 reals, row-major re, im), RP_REAL (4 reals: m00 m01 m10 m11; H, RY) or
                // RP_RX (4 reals: m00, Im m01, Im m10, m11; real diagonal, imaginary off-diagonal)
    RP_C1,      // the same, only where the bit at position a is 1
    RP_X,       // exchange on `slot` where the bit at position a is 1
    RP_DIAG,    // multiply by d[2 x_a + x_b] (one position: a = b, d1 = d2 unused)
    RP_NEG,     // negate where an odd number of slot + 1 patterns x_a x_b hold; the pairs
                // (a | b << 5) are payload reals 0..slot
    RP_PH,      // multiply by payload[0] + i payload[1] where x_a = x_b = 1; with slot field 1
                // (run form) a = nf one-position phases (position, re, im) and b = ns sign
                // pairs (a | b << 5): multiply by every phase whose position bit is 1, negate
                // where an odd number of pairs have both bits 1
    RP_PARITY,  // multiply by payload (0, 1) where x_a = x_b, by payload (2, 3) elsewhere
    RP_PARITYN, // np parity patterns (a | b << 5), then np + 1 factors (re, im) indexed by the
                // number of patterns with x_a != x_b (equal-angle RZZ / RZ layers), np <= 15
};
constexpr int kRpMaxParity = 15;
// Run form of RP_PH: at most 31 phases and 31 sign pairs (5-bit counts); below
// kRpMinRunPhases phases the separate members cost less.
constexpr int kRpMaxRunPhases = 31;
constexpr int kRpMaxRunPairs = 31;
constexpr int kRpMinRunPhases = 3;
// RP_R0: 7 reals (m00 real; m01, m10, m11 as re, im), only on slots whose bit of sigma is 0
// in every lane: positions 4 and up, with no exchange on the slot earlier in the phase (an
// exchange toggles the slot's bit of sigma), so the matrix is never conjugated
enum RpForm : int { RP_GENERAL = 0, RP_REAL = 1, RP_RX = 2, RP_R0 = 3 };

// Host+device description of one op in a given index space (HBM amplitude/element
// indices for K1, tile-local indices for K2).
struct KOp {
    int32_t fkind;
    int32_t nf;         // fixed bits (F_H..F_DENSE2)
    int32_t fb[3];      // fixed bits ascending
    int32_t nt;         // touched elements per group; F_CDIAGK: number of non-local terms
    uint64_t set_mask;  // forced-one bits
    uint64_t off[4];    // touched element offsets
    int32_t k;          // operand count (F_DIAGK / F_DENSEK); F_DENSE1: a D1_* structure class
    int32_t pos[8];     // operand positions, first = most significant (F_DIAGK / F_DENSEK)
    int32_t mat;        // offset of the op's reals in the parameter array
    int32_t nmat;       // number of reals
};

// KOp arrays are copied into shared memory in 4-byte words, followed by reals.
static_assert(sizeof(KOp) % 16 == 0, "KOp size keeps the reals after a KOp array aligned");

#ifdef __CUDACC__

template <typename T> struct C2T;
template <> struct C2T<double> { using type = double2; };
template <> struct C2T<float> { using type = float2; };

template <typename T, int L> struct Amp { T r[L], i[L]; };

// y = m0 * x0 + m1 * x1 (complex), 8 real multiply-adds.
template <typename T>
__device__ __forceinline__ void cdot2(T &yr, T &yi, T m0r, T m0i, T x0r, T x0i, T m1r, T m1i,
                                      T x1r, T x1i) {
    yr = m0r * x0r;
    yr = fma(-m0i, x0i, yr);
    yr = fma(m1r, x1r, yr);
    yr = fma(-m1i, x1i, yr);
    yi = m0r * x0i;
    yi = fma(m0i, x0r, yi);
    yi = fma(m1r, x1i, yi);
    yi = fma(m1i, x1r, yi);
}

// (a + b) r and (a - b) r as fma(r, a, +-r b): 3 floating-point instructions per real
// pair instead of 4 (the FP64 pipe is the limit for complex128 on this GPU).
template <typename T, int L>
__device__ __forceinline__ void f_h(Amp<T, L> *v, T r) {
#pragma unroll
    for (int l = 0; l < L; l++) {
        const T ar = v[0].r[l], ai = v[0].i[l];
        const T pr = r * v[1].r[l], pi = r * v[1].i[l];
        v[0].r[l] = fma(r, ar, pr); v[0].i[l] = fma(r, ai, pi);
        v[1].r[l] = fma(r, ar, -pr); v[1].i[l] = fma(r, ai, -pi);
    }
}
template <typename T, int L>
__device__ __forceinline__ void f_swap(Amp<T, L> *v) {
    const Amp<T, L> t = v[0];
    v[0] = v[1];
    v[1] = t;
}
template <typename T, int L>
__device__ __forceinline__ void f_dense1(Amp<T, L> *v, const T *m) {
#pragma unroll
    for (int l = 0; l < L; l++) {
        const T ar = v[0].r[l], ai = v[0].i[l], br = v[1].r[l], bi = v[1].i[l];
        cdot2(v[0].r[l], v[0].i[l], m[0], m[1], ar, ai, m[2], m[3], br, bi);
        cdot2(v[1].r[l], v[1].i[l], m[4], m[5], ar, ai, m[6], m[7], br, bi);
    }
}
// The same when m[0] has no imaginary part (U3, CU3, RX, RY: cos(theta/2) first): the first
// row takes 6 multiply-adds instead of 8, 7 per amplitude in all (complex128 U3 is bound
// by the FP64 pipe on this GPU).
template <typename T, int L>
__device__ __forceinline__ void f_dense1_r0(Amp<T, L> *v, const T *m) {
#pragma unroll
    for (int l = 0; l < L; l++) {
        const T ar = v[0].r[l], ai = v[0].i[l], br = v[1].r[l], bi = v[1].i[l];
        T pr = m[2] * br;
        pr = fma(-m[3], bi, pr);
        T pi = m[2] * bi;
        pi = fma(m[3], br, pi);
        cdot2(v[1].r[l], v[1].i[l], m[4], m[5], ar, ai, m[6], m[7], br, bi);
        v[0].r[l] = fma(m[0], ar, pr);
        v[0].i[l] = fma(m[0], ai, pi);
    }
}
// Real 2x2 (RY and other real rotations): 4 multiply-adds per amplitude.
template <typename T, int L>
__device__ __forceinline__ void f_dense1_real(Amp<T, L> *v, const T *m) {
#pragma unroll
    for (int l = 0; l < L; l++) {
        const T ar = v[0].r[l], ai = v[0].i[l], br = v[1].r[l], bi = v[1].i[l];
        v[0].r[l] = fma(m[0], ar, m[2] * br);
        v[0].i[l] = fma(m[0], ai, m[2] * bi);
        v[1].r[l] = fma(m[4], ar, m[6] * br);
        v[1].i[l] = fma(m[4], ai, m[6] * bi);
    }
}
// Real diagonal, imaginary off-diagonal (RX): 4 multiply-adds per amplitude.
template <typename T, int L>
__device__ __forceinline__ void f_dense1_rx(Amp<T, L> *v, const T *m) {
#pragma unroll
    for (int l = 0; l < L; l++) {
        const T ar = v[0].r[l], ai = v[0].i[l], br = v[1].r[l], bi = v[1].i[l];
        v[0].r[l] = fma(m[0], ar, -m[3] * bi);
        v[0].i[l] = fma(m[0], ai, m[3] * br);
        v[1].r[l] = fma(m[6], br, -m[5] * ai);
        v[1].i[l] = fma(m[6], bi, m[5] * ar);
    }
}
template <typename T, int L, int NT>
__device__ __forceinline__ void f_diag(Amp<T, L> *v, const T *d) {
#pragma unroll
    for (int t = 0; t < NT; t++)
#pragma unroll
        for (int l = 0; l < L; l++) {
            const T xr = v[t].r[l], xi = v[t].i[l];
            v[t].r[l] = fma(d[2 * t], xr, -d[2 * t + 1] * xi);
            v[t].i[l] = fma(d[2 * t], xi, d[2 * t + 1] * xr);
        }
}
template <typename T, int L>
__device__ __forceinline__ void f_neg(Amp<T, L> *v) {
#pragma unroll
    for (int l = 0; l < L; l++) {
        v[0].r[l] = -v[0].r[l];
        v[0].i[l] = -v[0].i[l];
    }
}
template <typename T, int L>
__device__ __forceinline__ void f_dense2(Amp<T, L> *v, const T *m) {
#pragma unroll
    for (int l = 0; l < L; l++) {
        T xr[4], xi[4];
#pragma unroll
        for (int t = 0; t < 4; t++) { xr[t] = v[t].r[l]; xi[t] = v[t].i[l]; }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            T yr, yi, zr, zi;
            cdot2(yr, yi, m[8 * r + 0], m[8 * r + 1], xr[0], xi[0], m[8 * r + 2], m[8 * r + 3], xr[1], xi[1]);
            cdot2(zr, zi, m[8 * r + 4], m[8 * r + 5], xr[2], xi[2], m[8 * r + 6], m[8 * r + 7], xr[3], xi[3]);
            v[r].r[l] = yr + zr;
            v[r].i[l] = yi + zi;
        }
    }
}

// Inserts a zero bit at each of the nf sorted positions fb[] of x (runtime nf <= 3).
__device__ __forceinline__ uint64_t insert_zero_bits(uint64_t x, int nf, const int32_t *fb) {
#pragma unroll
    for (int j = 0; j < 3; j++) {
        if (j < nf) {
            const int b = fb[j];
            x = ((x >> b) << (b + 1)) | (x & ((1ull << b) - 1ull));
        }
    }
    return x;
}

#endif  // __CUDACC__

}  // namespace qs
