// Applying a pass's ops to a tile held in shared memory (tile-local bit positions).
// Shared by the chunk kernel (K2) and the batched persistent kernel (K6).
#pragma once

#include <type_traits>

#include "dfmath.cuh"
#include "kops.cuh"

namespace qs {

constexpr int kMaxOpReals = 512;  // dense 4-qubit block: 2 * 16 * 16 reals

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
template <typename T> struct SDense2 {
    const T *m;
    __device__ void operator()(Amp<T, 1> *v) const { f_dense2<T, 1>(v, m); }
};
template <typename T, int NT> struct SDiag {
    const T *d;
    __device__ void operator()(Amp<T, 1> *v) const { f_diag<T, 1, NT>(v, d); }
};

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

// F_RGROUP (complex64): every thread owns groups of 16 amplitudes spanned by the 4
// positions pos[0..3] and applies a run of one- and two-bit ops to them in registers, one
// shared-memory sweep for the whole run.  Lane l keeps amplitude r ^ L (L = l & 15) in
// register r, so the 32 lanes of a warp touch different banks even when the 4 positions
// are the lowest ones; each member's matrix is read with its row and column indices XORed
// by L's bits on that member's positions, which is the same operator in that order.
// Block layout in sm: [member count, then per member: code, 2^(2 nb) complex entries],
// code = nb + 4 b0 + 16 b1 (nb in {1,2}; b0 < b1 register bits; sub-index s = bit b0 +
// 2 bit b1), entries row-major (re, im).
// Member matrices are copied into registers once per member, already permuted for this
// lane (entry (r, c) of the register copy is M[r ^ x][c ^ x]), so that the multiply-adds
// use uniform register operands.
template <int B0, int G>
__device__ __forceinline__ void rg_one(float2 (&v)[G][16], const float *M, int L) {
    const int x = (L >> B0) & 1;
    float m[8];
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int c = 0; c < 2; c++) {
            m[4 * r + 2 * c] = M[4 * (r ^ x) + 2 * (c ^ x)];
            m[4 * r + 2 * c + 1] = M[4 * (r ^ x) + 2 * (c ^ x) + 1];
        }
#pragma unroll
    for (int g = 0; g < G; g++)
#pragma unroll
        for (int r = 0; r < 16; r++) {
            if (r & (1 << B0)) continue;
            const float2 a = v[g][r], b = v[g][r | (1 << B0)];
#pragma unroll
            for (int so = 0; so < 2; so++) {
                const float *row = m + 4 * so;
                float yr = row[0] * a.x;
                yr = fmaf(-row[1], a.y, yr);
                yr = fmaf(row[2], b.x, yr);
                yr = fmaf(-row[3], b.y, yr);
                float yi = row[0] * a.y;
                yi = fmaf(row[1], a.x, yi);
                yi = fmaf(row[2], b.y, yi);
                yi = fmaf(row[3], b.x, yi);
                v[g][so ? (r | (1 << B0)) : r] = make_float2(yr, yi);
            }
        }
}
template <int B0, int B1, int G>
__device__ __forceinline__ void rg_two(float2 (&v)[G][16], const float *M, int L) {
    const int xm = ((L >> B0) & 1) | (((L >> B1) & 1) << 1);
    float m[32];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            m[8 * r + 2 * c] = M[8 * (r ^ xm) + 2 * (c ^ xm)];
            m[8 * r + 2 * c + 1] = M[8 * (r ^ xm) + 2 * (c ^ xm) + 1];
        }
#pragma unroll
    for (int g = 0; g < G; g++)
#pragma unroll
        for (int r = 0; r < 16; r++) {
            if (r & ((1 << B0) | (1 << B1))) continue;
            float2 a[4];
#pragma unroll
            for (int s = 0; s < 4; s++) a[s] = v[g][r | ((s & 1) << B0) | ((s >> 1) << B1)];
#pragma unroll
            for (int so = 0; so < 4; so++) {
                const float *row = m + 8 * so;
                float yr = 0.f, yi = 0.f;
#pragma unroll
                for (int s = 0; s < 4; s++) {
                    yr = fmaf(row[2 * s], a[s].x, yr);
                    yr = fmaf(-row[2 * s + 1], a[s].y, yr);
                    yi = fmaf(row[2 * s], a[s].y, yi);
                    yi = fmaf(row[2 * s + 1], a[s].x, yi);
                }
                v[g][r | ((so & 1) << B0) | ((so >> 1) << B1)] = make_float2(yr, yi);
            }
        }
}

// G groups of 16 per thread stay in registers while every member is applied.
template <int G>
__device__ __forceinline__ void rgroup_run(float2 *tile, const KOp &op, const float *sm, uint32_t g0, uint32_t gstep) {
    const uint32_t p0 = 1u << op.pos[0], p1 = 1u << op.pos[1], p2 = 1u << op.pos[2], p3 = 1u << op.pos[3];
    const int L = threadIdx.x & 15;
    const uint32_t dL = ((L & 1) ? p0 : 0u) | ((L & 2) ? p1 : 0u) | ((L & 4) ? p2 : 0u) | ((L & 8) ? p3 : 0u);
    float2 v[G][16];
    uint32_t base[G];
#pragma unroll
    for (int gi = 0; gi < G; gi++) {
        uint32_t b = g0 + gi * gstep;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int q = op.pos[j];
            b = ((b >> q) << (q + 1)) | (b & ((1u << q) - 1u));
        }
        base[gi] = b;
#pragma unroll
        for (int r = 0; r < 16; r++) {
            const uint32_t d = ((r & 1) ? p0 : 0u) | ((r & 2) ? p1 : 0u) | ((r & 4) ? p2 : 0u) | ((r & 8) ? p3 : 0u);
            v[gi][r] = tile[b | (d ^ dL)];
        }
    }
    const int nmem = (int)sm[0];
    int o = 1;
    for (int mi = 0; mi < nmem; mi++) {
        const int code = (int)sm[o];
        const float *M = sm + o + 1;
        if ((code & 3) == 1) {
            switch ((code >> 2) & 3) {
            case 0: rg_one<0, G>(v, M, L); break;
            case 1: rg_one<1, G>(v, M, L); break;
            case 2: rg_one<2, G>(v, M, L); break;
            default: rg_one<3, G>(v, M, L); break;
            }
            o += 9;
        } else {
            switch (code >> 2) {
            case 0 + 4 * 1: rg_two<0, 1, G>(v, M, L); break;
            case 0 + 4 * 2: rg_two<0, 2, G>(v, M, L); break;
            case 0 + 4 * 3: rg_two<0, 3, G>(v, M, L); break;
            case 1 + 4 * 2: rg_two<1, 2, G>(v, M, L); break;
            case 1 + 4 * 3: rg_two<1, 3, G>(v, M, L); break;
            default: rg_two<2, 3, G>(v, M, L); break;
            }
            o += 33;
        }
    }
#pragma unroll
    for (int gi = 0; gi < G; gi++)
#pragma unroll
        for (int r = 0; r < 16; r++) {
            const uint32_t d = ((r & 1) ? p0 : 0u) | ((r & 2) ? p1 : 0u) | ((r & 4) ? p2 : 0u) | ((r & 8) ? p3 : 0u);
            tile[base[gi] | (d ^ dL)] = v[gi][r];
        }
}

__device__ __forceinline__ void rgroup_apply(float2 *tile, const KOp &op, const float *sm, int m) {
    const uint32_t ng = 1u << (m - 4);
    if (ng == 2u * blockDim.x) {
        rgroup_run<2>(tile, op, sm, threadIdx.x, blockDim.x);
    } else {
        for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) rgroup_run<1>(tile, op, sm, g, 0);
    }
}

// Applies one op to the tile; op and its matrix entries are in shared memory.
template <typename T>
__device__ __forceinline__ void apply_op_smem(typename C2T<T>::type *tile, const KOp &op, const T *sm, int m) {
    switch (op.fkind) {
    case F_H: groups_apply<T, 2>(tile, op, m, SH<T>{(T)0.70710678118654752440}); break;
    case F_SWAP: groups_apply<T, 2>(tile, op, m, SSwap<T>{}); break;
    case F_DENSE1: groups_apply<T, 2>(tile, op, m, SDense1<T>{sm}); break;
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
    case F_DENSEK:
        if (op.k == 3) dense_k_smem<T, 3>(tile, op, sm, m);
        else if (op.k == 4) dense_k_smem<T, 4>(tile, op, sm, m);
        break;
    case F_RGROUP:
        if constexpr (std::is_same<T, float>::value) rgroup_apply(tile, op, sm, m);
        break;
    default:
        break;
    }
}

// ---- complex128 ops with double-float arithmetic (matrix reals as (hi, lo) pairs) --------
__device__ __forceinline__ df::F2 dfneg(df::F2 a) { return df::F2{-a.h, -a.l}; }

struct SDfH {
    df::F2 r;
    __device__ void operator()(Amp<double, 1> *v) const {
        const df::F2 ar = df::split(v[0].r[0]), ai = df::split(v[0].i[0]);
        const df::F2 br = df::split(v[1].r[0]), bi = df::split(v[1].i[0]);
        v[0].r[0] = df::result(df::scale(df::add(ar, br), r));
        v[0].i[0] = df::result(df::scale(df::add(ai, bi), r));
        v[1].r[0] = df::result(df::scale(df::sub(ar, br), r));
        v[1].i[0] = df::result(df::scale(df::sub(ai, bi), r));
    }
};
// y_r = sum_c m[r][c] x_c over NT touched elements, matrix as pairs (row-major, re/im)
template <int NT> struct SDfDense {
    const df::F2 *m;
    __device__ void operator()(Amp<double, 1> *v) const {
        df::F2 xr[NT], xi[NT];
#pragma unroll
        for (int t = 0; t < NT; t++) {
            xr[t] = df::split(v[t].r[0]);
            xi[t] = df::split(v[t].i[0]);
        }
#pragma unroll
        for (int r = 0; r < NT; r++) {
            const df::F2 *row = m + 2 * NT * r;
            df::Acc a = df::mul(row[0], xr[0]);
            df::Acc b = df::mul(row[0], xi[0]);
            df::mac(a, dfneg(row[1]), xi[0]);
            df::mac(b, row[1], xr[0]);
#pragma unroll
            for (int c = 1; c < NT; c++) {
                df::mac(a, row[2 * c], xr[c]);
                df::mac(a, dfneg(row[2 * c + 1]), xi[c]);
                df::mac(b, row[2 * c], xi[c]);
                df::mac(b, row[2 * c + 1], xr[c]);
            }
            v[r].r[0] = df::result(a);
            v[r].i[0] = df::result(b);
        }
    }
};
template <int NT> struct SDfDiag {
    const df::F2 *d;
    __device__ void operator()(Amp<double, 1> *v) const {
#pragma unroll
        for (int t = 0; t < NT; t++) {
            const df::F2 xr = df::split(v[t].r[0]), xi = df::split(v[t].i[0]);
            df::Acc a = df::mul(d[2 * t], xr);
            df::mac(a, dfneg(d[2 * t + 1]), xi);
            df::Acc b = df::mul(d[2 * t], xi);
            df::mac(b, d[2 * t + 1], xr);
            v[t].r[0] = df::result(a);
            v[t].i[0] = df::result(b);
        }
    }
};

// Applies one op with double-float arithmetic; sm holds the op's reals as (hi, lo) pairs.
// Wider diagonal and dense blocks rebuild FP64 entries (hi + lo) and use FP64 arithmetic.
__device__ __forceinline__ void apply_op_smem_df(double2 *tile, const KOp &op, const df::F2 *sm, double *sd,
                                                 int m) {
    switch (op.fkind) {
    case F_H: groups_apply<double, 2>(tile, op, m, SDfH{df::F2{0.70710677f, 1.21016175e-08f}}); break;
    case F_SWAP: groups_apply<double, 2>(tile, op, m, SSwap<double>{}); break;
    case F_NEG: groups_apply<double, 1>(tile, op, m, SNeg<double>{}); break;
    case F_DENSE1: groups_apply<double, 2>(tile, op, m, SDfDense<2>{sm}); break;
    case F_DIAG1: groups_apply<double, 2>(tile, op, m, SDfDiag<2>{sm}); break;
    case F_PHASE: groups_apply<double, 1>(tile, op, m, SDfDiag<1>{sm}); break;
    case F_DIAG2: groups_apply<double, 4>(tile, op, m, SDfDiag<4>{sm}); break;
    case F_DENSE2: groups_apply<double, 4>(tile, op, m, SDfDense<4>{sm}); break;
    default: {
        for (int j = threadIdx.x; j < op.nmat; j += blockDim.x) sd[j] = (double)sm[j].h + (double)sm[j].l;
        __syncthreads();
        apply_op_smem<double>(tile, op, sd, m);
        break;
    }
    }
}

// Stages op i and its matrix entries into shared memory, then applies it; every thread
// of the block must call this (it synchronises).
template <typename T>
__device__ __forceinline__ void apply_ops_tile(typename C2T<T>::type *tile, const KOp *ops, int n_ops,
                                               const T *mats, int m, KOp &s_op, T *s_m) {
    for (int i = 0; i < n_ops; i++) {
        if (threadIdx.x == 0) s_op = ops[i];
        __syncthreads();
        for (int j = threadIdx.x; j < s_op.nmat; j += blockDim.x) s_m[j] = mats[s_op.mat + j];
        __syncthreads();
        apply_op_smem<T>(tile, s_op, s_m, m);
        __syncthreads();
    }
}

}  // namespace qs
