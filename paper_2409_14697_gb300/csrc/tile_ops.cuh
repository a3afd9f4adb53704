// Applying a pass's ops to a tile held in shared memory (tile-local bit positions).
// Shared by the chunk kernel (K2) and the batched persistent kernel (K6).
#pragma once

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
