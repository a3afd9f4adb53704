// K1: streaming gate kernels — one gate, one pass over the state vector in HBM.
//
// QueenV2 (arXiv 2409.14697) Sec. II-A: Eq. 2 updates every pair of amplitudes that
// differ only in the target bit; Eq. 3 updates every group of four selected by two bits
// (CNOT: first operand = control); a k-qubit gate updates every group of 2^k.  Each
// thread owns U groups at once (all loads issued before any arithmetic, so that every
// thread keeps 2*U 16-byte loads in flight), consecutive threads own consecutive
// groups (coalesced along the low bits), and the grid is a persistent multiple of the
// SM count.  Only the amplitudes a gate changes are touched: CNOT/SWAP/CU3 read and
// write half the vector, CZ/CP a quarter.
//
// Element types: complex128 = double2 (16 B, one amplitude); complex64 = float4 (two
// consecutive amplitudes, used when every fixed bit is >= 1, so the element index is the
// amplitude index >> 1) or float2 (one amplitude, when bit 0 is a gate operand).
#include <algorithm>
#include <mutex>
#include <map>
#include <tuple>
#include <type_traits>

#include "dfmath.cuh"
#include "ixmath.cuh"
#include "kgeom.h"
#include "kops.cuh"
#include "qs_internal.h"

namespace qs {
namespace {

template <typename T, int L> struct VecT;
template <> struct VecT<double, 1> { using type = double2; };
template <> struct VecT<float, 1> { using type = float2; };
template <> struct VecT<float, 2> { using type = float4; };

__device__ __forceinline__ void ldv(const double2 *p, Amp<double, 1> &a) {
    const double2 v = *p;
    a.r[0] = v.x; a.i[0] = v.y;
}
__device__ __forceinline__ void ldv(const float2 *p, Amp<float, 1> &a) {
    const float2 v = *p;
    a.r[0] = v.x; a.i[0] = v.y;
}
__device__ __forceinline__ void ldv(const float4 *p, Amp<float, 2> &a) {
    const float4 v = *p;
    a.r[0] = v.x; a.i[0] = v.y; a.r[1] = v.z; a.i[1] = v.w;
}
__device__ __forceinline__ void stv(double2 *p, const Amp<double, 1> &a) { *p = make_double2(a.r[0], a.i[0]); }
__device__ __forceinline__ void stv(float2 *p, const Amp<float, 1> &a) { *p = make_float2(a.r[0], a.i[0]); }
__device__ __forceinline__ void stv(float4 *p, const Amp<float, 2> &a) {
    *p = make_float4(a.r[0], a.i[0], a.r[1], a.i[1]);
}

// ---- functors (matrix entries by value in the kernel parameters) ----------------
template <typename T> struct FH {
    static constexpr int NT = 2;
    T r;
    template <int L> __device__ void operator()(Amp<T, L> *v) const { f_h<T, L>(v, r); }
};
// The Hadamard butterfly without its scale (a + b, a - b): 2 additions per amplitude.
template <typename T> struct FHSum {
    static constexpr int NT = 2;
    template <int L> __device__ void operator()(Amp<T, L> *v) const {
#pragma unroll
        for (int l = 0; l < L; l++) {
            const T ar = v[0].r[l], ai = v[0].i[l], br = v[1].r[l], bi = v[1].i[l];
            v[0].r[l] = ar + br; v[0].i[l] = ai + bi;
            v[1].r[l] = ar - br; v[1].i[l] = ai - bi;
        }
    }
};
template <typename T> struct FSwap {
    static constexpr int NT = 2;
    template <int L> __device__ void operator()(Amp<T, L> *v) const { f_swap<T, L>(v); }
};
template <typename T> struct FDense1 {
    static constexpr int NT = 2;
    T m[8];
    template <int L> __device__ void operator()(Amp<T, L> *v) const { f_dense1<T, L>(v, m); }
};
template <typename T> struct FDense1R0 {
    static constexpr int NT = 2;
    T m[8];
    template <int L> __device__ void operator()(Amp<T, L> *v) const { f_dense1_r0<T, L>(v, m); }
};
template <typename T> struct FDense1Real {
    static constexpr int NT = 2;
    T m[8];
    template <int L> __device__ void operator()(Amp<T, L> *v) const { f_dense1_real<T, L>(v, m); }
};
template <typename T> struct FDense1RX {
    static constexpr int NT = 2;
    T m[8];
    template <int L> __device__ void operator()(Amp<T, L> *v) const { f_dense1_rx<T, L>(v, m); }
};
template <typename T> struct FDiag1 {
    static constexpr int NT = 2;
    T d[4];
    template <int L> __device__ void operator()(Amp<T, L> *v) const { f_diag<T, L, 2>(v, d); }
};
template <typename T> struct FPhase {
    static constexpr int NT = 1;
    T d[2];
    template <int L> __device__ void operator()(Amp<T, L> *v) const { f_diag<T, L, 1>(v, d); }
};
template <typename T> struct FNeg {
    static constexpr int NT = 1;
    template <int L> __device__ void operator()(Amp<T, L> *v) const { f_neg<T, L>(v); }
};
template <typename T> struct FDiag2 {
    static constexpr int NT = 4;
    T d[8];
    template <int L> __device__ void operator()(Amp<T, L> *v) const { f_diag<T, L, 4>(v, d); }
};
template <typename T> struct FDense2 {
    static constexpr int NT = 4;
    T m[32];
    template <int L> __device__ void operator()(Amp<T, L> *v) const { f_dense2<T, L>(v, m); }
};

// ---- complex128 functors with double-float (FP32 pair) arithmetic ---------------
// Matrix entries arrive as (hi, lo) float pairs split on the host; amplitudes are split
// and re-joined in the kernel (dfmath.cuh).  Same group structure as the FP64 functors.
using df::F2;

__device__ __forceinline__ F2 neg(F2 a) { return F2{-a.h, -a.l}; }

// y = m0 * x0 + m1 * x1, complex, compensated
__device__ __forceinline__ void df_cdot2(double &yr, double &yi, const F2 *m0, F2 x0r, F2 x0i, const F2 *m1,
                                         F2 x1r, F2 x1i) {
    df::Acc a = df::mul(m0[0], x0r);
    df::mac(a, neg(m0[1]), x0i);
    df::mac(a, m1[0], x1r);
    df::mac(a, neg(m1[1]), x1i);
    df::Acc b = df::mul(m0[0], x0i);
    df::mac(b, m0[1], x0r);
    df::mac(b, m1[0], x1i);
    df::mac(b, m1[1], x1r);
    yr = df::result(a);
    yi = df::result(b);
}

// y = d * x, complex, compensated
__device__ __forceinline__ void df_cmul(double &yr, double &yi, const F2 *d, F2 xr, F2 xi) {
    df::Acc a = df::mul(d[0], xr);
    df::mac(a, neg(d[1]), xi);
    df::Acc b = df::mul(d[0], xi);
    df::mac(b, d[1], xr);
    yr = df::result(a);
    yi = df::result(b);
}

struct FHDF {
    static constexpr int NT = 2;
    F2 r;
    template <int L> __device__ void operator()(Amp<double, L> *v) const {
        const F2 ar = df::split(v[0].r[0]), ai = df::split(v[0].i[0]);
        const F2 br = df::split(v[1].r[0]), bi = df::split(v[1].i[0]);
        v[0].r[0] = df::result(df::scale(df::add(ar, br), r));
        v[0].i[0] = df::result(df::scale(df::add(ai, bi), r));
        v[1].r[0] = df::result(df::scale(df::sub(ar, br), r));
        v[1].i[0] = df::result(df::scale(df::sub(ai, bi), r));
    }
};
struct FDense1DF {
    static constexpr int NT = 2;
    F2 m[8];
    template <int L> __device__ void operator()(Amp<double, L> *v) const {
        const F2 x0r = df::split(v[0].r[0]), x0i = df::split(v[0].i[0]);
        const F2 x1r = df::split(v[1].r[0]), x1i = df::split(v[1].i[0]);
        df_cdot2(v[0].r[0], v[0].i[0], m + 0, x0r, x0i, m + 2, x1r, x1i);
        df_cdot2(v[1].r[0], v[1].i[0], m + 4, x0r, x0i, m + 6, x1r, x1i);
    }
};
template <int NTT> struct FDiagDF {
    static constexpr int NT = NTT;
    F2 d[2 * NTT];
    template <int L> __device__ void operator()(Amp<double, L> *v) const {
#pragma unroll
        for (int t = 0; t < NTT; t++) {
            const F2 xr = df::split(v[t].r[0]), xi = df::split(v[t].i[0]);
            df_cmul(v[t].r[0], v[t].i[0], d + 2 * t, xr, xi);
        }
    }
};
struct FDense2DF {
    static constexpr int NT = 4;
    F2 m[32];
    template <int L> __device__ void operator()(Amp<double, L> *v) const {
        F2 xr[4], xi[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            xr[t] = df::split(v[t].r[0]);
            xi[t] = df::split(v[t].i[0]);
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const F2 *row = m + 8 * r;
            df::Acc a = df::mul(row[0], xr[0]);
            df::Acc b = df::mul(row[0], xi[0]);
            df::mac(a, neg(row[1]), xi[0]);
            df::mac(b, row[1], xr[0]);
#pragma unroll
            for (int c = 1; c < 4; c++) {
                df::mac(a, row[2 * c], xr[c]);
                df::mac(a, neg(row[2 * c + 1]), xi[c]);
                df::mac(b, row[2 * c], xi[c]);
                df::mac(b, row[2 * c + 1], xr[c]);
            }
            v[r].r[0] = df::result(a);
            v[r].i[0] = df::result(b);
        }
    }
};

// ---- complex128 functors with integer products (ixmath.cuh) ----------------------
// Each real output is one ix::dot over its terms, with the matrix entries decoded on the
// host (ix::rows_dense1 / ix::rows_diag, signs included).  The first NAT of a thread's
// groups take the native FP64 functor instead, so the FP64 pipe and the integer pipes
// work side by side.
__device__ __forceinline__ void ix_pair(const Amp<double, 1> *v, ix::Num (&x)[4]) {
    x[0] = ix::decode(v[0].r[0]);
    x[1] = ix::decode(v[0].i[0]);
    x[2] = ix::decode(v[1].r[0]);
    x[3] = ix::decode(v[1].i[0]);
}
__device__ __forceinline__ void ix_store(Amp<double, 1> *v, const double (&y)[4]) {
    v[0].r[0] = y[0]; v[0].i[0] = y[1];
    v[1].r[0] = y[2]; v[1].i[0] = y[3];
}

// U3 / CU3 (Im m00 = 0): 14 terms
template <int ENC, int UG, int NAT, int MB> struct FDense1R0IX {
    static constexpr int NT = 2;
    static constexpr int kGroups = UG;
    static constexpr int kNative = NAT;
    static constexpr int kMinBlocks = MB;
    ix::Num c[14];
    double m[8];
    template <int L> __device__ void operator()(Amp<double, L> *v) const {
        ix::Num x[4];
        double y[4];
        ix_pair(v, x);
        ix::dense1_r0<ENC>(c, x, y);
        ix_store(v, y);
    }
    template <int L> __device__ void native(Amp<double, L> *v) const { f_dense1_r0<double, L>(v, m); }
};

// general 2x2: 16 terms
template <int ENC, int UG, int NAT, int MB> struct FDense1IX {
    static constexpr int NT = 2;
    static constexpr int kGroups = UG;
    static constexpr int kNative = NAT;
    static constexpr int kMinBlocks = MB;
    ix::Num c[16];
    double m[8];
    template <int L> __device__ void operator()(Amp<double, L> *v) const {
        ix::Num x[4];
        double y[4];
        ix_pair(v, x);
        ix::dense1<ENC>(c, x, y);
        ix_store(v, y);
    }
    template <int L> __device__ void native(Amp<double, L> *v) const { f_dense1<double, L>(v, m); }
};

// real 2x2 (RY) and RX forms: rows of 2 terms
template <int ENC, int UG, int NAT, int MB> struct FDense1RealIX {
    static constexpr int NT = 2;
    static constexpr int kGroups = UG;
    static constexpr int kNative = NAT;
    static constexpr int kMinBlocks = MB;
    ix::Num c[8];
    double m[8];
    template <int L> __device__ void operator()(Amp<double, L> *v) const {
        ix::Num x[4];
        double y[4];
        ix_pair(v, x);
        ix::dense1_real<ENC>(c, x, y);
        ix_store(v, y);
    }
    template <int L> __device__ void native(Amp<double, L> *v) const { f_dense1_real<double, L>(v, m); }
};
template <int ENC, int UG, int NAT, int MB> struct FDense1RXIX {
    static constexpr int NT = 2;
    static constexpr int kGroups = UG;
    static constexpr int kNative = NAT;
    static constexpr int kMinBlocks = MB;
    ix::Num c[8];
    double m[8];
    template <int L> __device__ void operator()(Amp<double, L> *v) const {
        ix::Num x[4];
        double y[4];
        ix_pair(v, x);
        ix::dense1_rx<ENC>(c, x, y);
        ix_store(v, y);
    }
    template <int L> __device__ void native(Amp<double, L> *v) const { f_dense1_rx<double, L>(v, m); }
};

// diagonal: NTT elements, each times its own factor
template <int ENC, int NTT, int UG, int NAT, int MB> struct FDiagIX {
    static constexpr int NT = NTT;
    static constexpr int kGroups = UG;
    static constexpr int kNative = NAT;
    static constexpr int kMinBlocks = MB;
    ix::Num c[4 * NTT];
    double d[2 * NTT];
    template <int L> __device__ void operator()(Amp<double, L> *v) const {
#pragma unroll
        for (int t = 0; t < NTT; t++) {
            const ix::Num x[2] = {ix::decode(v[t].r[0]), ix::decode(v[t].i[0])};
            double y[2];
            ix::phase<ENC>(c + 4 * t, x, y);
            v[t].r[0] = y[0];
            v[t].i[0] = y[1];
        }
    }
    template <int L> __device__ void native(Amp<double, L> *v) const { f_diag<double, L, NTT>(v, d); }
};

void split_host(double v, F2 &o) {
    o.h = (float)v;
    o.l = (float)(v - (double)o.h);
}

constexpr int kThreads = 256;

struct Geom {
    int32_t fb[3];
    uint64_t set_mask;
    uint64_t off[4];
    uint64_t n_groups;
};

template <int NF>
__device__ __forceinline__ uint64_t insert_zeros(uint64_t x, const Geom &g) {
#pragma unroll
    for (int j = 0; j < NF; j++) {
        const int b = g.fb[j];
        x = ((x >> b) << (b + 1)) | (x & ((1ull << b) - 1ull));
    }
    return x;
}

// Functors with integer products may give their first kNative groups per thread to the
// native FP64 form.
template <typename F, typename = void> struct NativeGroups { static constexpr int value = 0; };
template <typename F> struct NativeGroups<F, std::void_t<decltype(F::kNative)>> {
    static constexpr int value = F::kNative;
};

// Resident CTAs per SM the compiler must allow (register cap), if the functor sets one.
template <typename F, typename = void> struct MinBlocks { static constexpr int value = 1; };
template <typename F> struct MinBlocks<F, std::void_t<decltype(F::kMinBlocks)>> {
    static constexpr int value = F::kMinBlocks;
};

template <typename T, int L, int NF, int U, typename F>
__global__ void __launch_bounds__(kThreads, MinBlocks<F>::value)
k_stream(typename VecT<T, L>::type *__restrict__ psi, const Geom g, const F f) {
    constexpr int NT = F::NT;
    const uint64_t per_iter = (uint64_t)kThreads * U;
    for (uint64_t b0 = (uint64_t)blockIdx.x * per_iter; b0 < g.n_groups; b0 += (uint64_t)gridDim.x * per_iter) {
        Amp<T, L> v[U][NT];
        uint64_t base[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint64_t gi = b0 + (uint64_t)u * kThreads + threadIdx.x;
            base[u] = insert_zeros<NF>(gi, g) | g.set_mask;
            if (gi < g.n_groups) {
#pragma unroll
                for (int t = 0; t < NT; t++) ldv(psi + (base[u] + g.off[t]), v[u][t]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (b0 + (uint64_t)u * kThreads + threadIdx.x < g.n_groups) {
                if constexpr (NativeGroups<F>::value > 0) {
                    if (u < NativeGroups<F>::value) f.native(v[u]);
                    else f(v[u]);
                } else {
                    f(v[u]);
                }
            }
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (b0 + (uint64_t)u * kThreads + threadIdx.x < g.n_groups) {
#pragma unroll
                for (int t = 0; t < NT; t++) stv(psi + (base[u] + g.off[t]), v[u][t]);
            }
        }
    }
}

// Diagonal on k >= 3 qubits: every amplitude times d[sub-index of its operand bits].
template <typename T, int L>
__global__ void __launch_bounds__(kThreads)
k_diag_general(typename VecT<T, L>::type *__restrict__ psi, uint64_t n_elem, int k, int4 qa, int4 qb,
               const T *__restrict__ d) {
    const int q[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
    for (uint64_t e = (uint64_t)blockIdx.x * kThreads + threadIdx.x; e < n_elem; e += (uint64_t)gridDim.x * kThreads) {
        Amp<T, L> a;
        ldv(psi + e, a);
#pragma unroll
        for (int l = 0; l < L; l++) {
            const uint64_t x = e * L + l;
            uint32_t s = 0;
            for (int j = 0; j < k; j++) s |= (uint32_t)((x >> q[j]) & 1ull) << (k - 1 - j);
            const T c = d[2 * s], sn = d[2 * s + 1];
            const T xr = a.r[l], xi = a.i[l];
            a.r[l] = fma(c, xr, -sn * xi);
            a.i[l] = fma(c, xi, sn * xr);
        }
        stv(psi + e, a);
    }
}

// Dense k-qubit block on SIMT (k = 3..6): one thread per group of 2^k amplitudes.
template <typename T, int K>
__global__ void __launch_bounds__(128)
k_dense_general(typename VecT<T, 1>::type *__restrict__ psi, uint64_t n_groups, int4 qa, int4 qb,
                const T *__restrict__ m) {
    constexpr int D = 1 << K;
    __shared__ uint64_t soff[D];
    __shared__ int sorted_s[8];
    const int q[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
    if (threadIdx.x == 0) {
        int s[8];
        for (int j = 0; j < K; j++) s[j] = q[j];
        for (int a = 1; a < K; a++)
            for (int b = a; b > 0 && s[b - 1] > s[b]; b--) {
                const int t = s[b]; s[b] = s[b - 1]; s[b - 1] = t;
            }
        for (int j = 0; j < K; j++) sorted_s[j] = s[j];
    }
    for (int s = threadIdx.x; s < D; s += blockDim.x) {
        uint64_t o = 0;
        for (int j = 0; j < K; j++) o |= (uint64_t)((s >> (K - 1 - j)) & 1) << q[j];
        soff[s] = o;
    }
    __syncthreads();
    for (uint64_t gi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < n_groups;
         gi += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x = gi;
#pragma unroll
        for (int j = 0; j < K; j++) {
            const int b = sorted_s[j];
            x = ((x >> b) << (b + 1)) | (x & ((1ull << b) - 1ull));
        }
        T vr[D], vi[D];
#pragma unroll
        for (int s = 0; s < D; s++) {
            Amp<T, 1> a;
            ldv(psi + x + soff[s], a);
            vr[s] = a.r[0]; vi[s] = a.i[0];
        }
#pragma unroll 1
        for (int r = 0; r < D; r++) {
            T yr = 0, yi = 0;
#pragma unroll
            for (int c = 0; c < D; c++) {
                const T mr = m[2 * (r * D + c)], mi = m[2 * (r * D + c) + 1];
                yr = fma(mr, vr[c], yr);
                yr = fma(-mi, vi[c], yr);
                yi = fma(mr, vi[c], yi);
                yi = fma(mi, vr[c], yi);
            }
            Amp<T, 1> o;
            o.r[0] = yr; o.i[0] = yi;
            stv(psi + x + soff[r], o);
        }
    }
}

// Groups per thread: 2, 4 or 8 by touched elements, unless the functor sets kGroups.
template <typename F, typename = void> struct GroupsPerThread {
    static constexpr int value = F::NT == 4 ? 2 : (F::NT == 2 ? 4 : 8);
};
template <typename F> struct GroupsPerThread<F, std::void_t<decltype(F::kGroups)>> {
    static constexpr int value = F::kGroups;
};

template <typename T, int L, int NF, typename F>
void run(DeviceState &st, const Geom &g, const F &f) {
    constexpr int U = GroupsPerThread<F>::value;
    auto kern = k_stream<T, L, NF, U, F>;
    const uint64_t per_iter = (uint64_t)kThreads * U;
    const int grid = persistent_grid((const void *)kern, kThreads, 0, (g.n_groups + per_iter - 1) / per_iter);
    kern<<<grid, kThreads, 0, st.stream>>>((typename VecT<T, L>::type *)st.psi, g, f);
    QS_CUDA(cudaGetLastError());
    count_launch();
}

template <typename T, int L, typename F>
void run_nf(DeviceState &st, int nf, const Geom &g, const F &f) {
    if (nf == 1) run<T, L, 1>(st, g, f);
    else if (nf == 2) run<T, L, 2>(st, g, f);
    else fail(QS_ERR_INVALID, "streaming op with unsupported fixed-bit count");
}

// Element geometry: float4 elements (two amplitudes) when the dtype is complex64 and no
// fixed bit is bit 0 (element index = amplitude index >> 1).
template <typename T, typename F>
void dispatch_elem(DeviceState &st, const KOp &k, const F &f) {
    Geom g{};
    for (int j = 0; j < k.nf; j++) g.fb[j] = k.fb[j];
    g.set_mask = k.set_mask;
    for (int t = 0; t < k.nt; t++) g.off[t] = k.off[t];
    g.n_groups = 1ull << (st.n - k.nf);
    if constexpr (std::is_same<T, double>::value) {
        run_nf<T, 1>(st, k.nf, g, f);
    } else if (k.fb[0] >= 1) {
        for (int j = 0; j < k.nf; j++) g.fb[j] -= 1;
        g.set_mask >>= 1;
        for (int t = 0; t < k.nt; t++) g.off[t] >>= 1;
        g.n_groups >>= 1;
        run_nf<float, 2>(st, k.nf, g, f);
    } else {
        run_nf<float, 1>(st, k.nf, g, f);
    }
}

template <typename T>
void load_m(T *dst, const std::vector<double> &mats, const KOp &k) {
    for (int i = 0; i < k.nmat; i++) dst[i] = (T)mats[k.mat + i];
}

template <typename F, int N>
void load_pairs(F &f, F2 (&dst)[N], const std::vector<double> &mats, const KOp &k) {
    for (int i = 0; i < k.nmat && i < N; i++) split_host(mats[k.mat + i], dst[i]);
}

// complex128 with double-float arithmetic; returns false for kinds it does not cover
bool launch_df(DeviceState &st, const KOp &k, const std::vector<double> &mats) {
    switch (k.fkind) {
    case F_H: {
        FHDF f;
        split_host(k.nmat ? mats[k.mat] : 1.0 / std::sqrt(2.0), f.r);
        dispatch_elem<double>(st, k, f);
        return true;
    }
    case F_DENSE1: { FDense1DF f; load_pairs(f, f.m, mats, k); dispatch_elem<double>(st, k, f); return true; }
    case F_DIAG1: { FDiagDF<2> f; load_pairs(f, f.d, mats, k); dispatch_elem<double>(st, k, f); return true; }
    case F_PHASE: { FDiagDF<1> f; load_pairs(f, f.d, mats, k); dispatch_elem<double>(st, k, f); return true; }
    case F_DIAG2: { FDiagDF<4> f; load_pairs(f, f.d, mats, k); dispatch_elem<double>(st, k, f); return true; }
    case F_DENSE2: { FDense2DF f; load_pairs(f, f.m, mats, k); dispatch_elem<double>(st, k, f); return true; }
    default: return false;
    }
}

// complex128 with integer products (QS_PREC_IX64); false for kinds it does not cover.
template <int E2, int U2, int N2, int E1, int U1, int N1, int MB1, int MB2>
bool launch_ix_t(DeviceState &st, const KOp &k, const std::vector<double> &mats) {
    switch (k.fkind) {
    case F_DENSE1: {
        double m[8];
        for (int i = 0; i < 8; i++) m[i] = mats[k.mat + i];
        if (k.k == D1_REAL) {
            FDense1RealIX<E2, U2, N2, MB2> f;
            ix::rows_dense1_real(f.c, m);
            std::copy(m, m + 8, f.m);
            dispatch_elem<double>(st, k, f);
        } else if (k.k == D1_RX) {
            FDense1RXIX<E2, U2, N2, MB2> f;
            ix::rows_dense1_rx(f.c, m);
            std::copy(m, m + 8, f.m);
            dispatch_elem<double>(st, k, f);
        } else if (k.k == D1_R0) {
            FDense1R0IX<E2, U2, N2, MB2> f;
            ix::rows_dense1(f.c, m, true);
            std::copy(m, m + 8, f.m);
            dispatch_elem<double>(st, k, f);
        } else {
            FDense1IX<E2, U2, N2, MB2> f;
            ix::rows_dense1(f.c, m, false);
            std::copy(m, m + 8, f.m);
            dispatch_elem<double>(st, k, f);
        }
        return true;
    }
    case F_PHASE: {
        FDiagIX<E1, 1, U1, N1, MB1> f;
        for (int i = 0; i < 2; i++) f.d[i] = mats[k.mat + i];
        ix::rows_diag(f.c, f.d, 1);
        dispatch_elem<double>(st, k, f);
        return true;
    }
    case F_DIAG1: {
        FDiagIX<E2, 2, U2, N2, MB2> f;
        for (int i = 0; i < 4; i++) f.d[i] = mats[k.mat + i];
        ix::rows_diag(f.c, f.d, 2);
        dispatch_elem<double>(st, k, f);
        return true;
    }
    default: return false;
    }
}

// Two-element kernels: 4 groups per thread, the first in native FP64; phases (one element):
// 6 groups per thread, the first in native FP64, at most 64 registers (4 CTAs of 256
// threads per SM).
// Every output through the conversion instruction.  Measured at 28 qubits on the GB300:
// U3 1.84 ms against 3.60 ms native, CU3 0.98 / 1.81, RZ phase 0.76 / 1.09, RY and RX
// 1.33 / 2.08.  With all groups in integer form, 3-6 groups per thread with 1-2 native,
// 3-4 CTAs per SM, or half or all of the outputs encoded with integer instructions (less
// FP64-pipe work), each was 2-10 % slower: the FP64 pipe is 71 % busy and instruction
// issue 50 % (ncu), the rest is dependency latency.
bool launch_ix(DeviceState &st, const KOp &k, const std::vector<double> &mats) {
    return launch_ix_t<0, 4, 1, 0, 6, 1, 4, 1>(st, k, mats);
}

template <typename T>
void launch_typed(DeviceState &st, const Op &op) {
    const int n = st.n;
    std::vector<int> ident(64);
    for (int i = 0; i < 64; i++) ident[i] = i;
    std::vector<double> mats;
    const KOp k = make_kop(op, ident.data(), mats);
    if constexpr (std::is_same<T, double>::value) {
        if (st.prec == QS_PREC_DF32 && launch_df(st, k, mats)) return;
        if (st.ix && launch_ix(st, k, mats)) return;
    }
    switch (k.fkind) {
    case F_H: {
        const double r = k.nmat ? mats[k.mat] : 1.0 / std::sqrt(2.0);
        if (r == 1.0) {
            dispatch_elem<T>(st, k, FHSum<T>{});
            return;
        }
        FH<T> f;
        f.r = (T)r;
        dispatch_elem<T>(st, k, f);
        return;
    }
    case F_SWAP: dispatch_elem<T>(st, k, FSwap<T>{}); return;
    case F_NEG: dispatch_elem<T>(st, k, FNeg<T>{}); return;
    case F_DENSE1: {
        // complex128 is bound by the FP64 pipe: use the cheapest form the matrix allows
        // (complex64 is bound by HBM, every form takes the same time)
        const int cls = std::is_same<T, double>::value ? k.k : (int)D1_GENERAL;
        if (cls == D1_REAL) {
            FDense1Real<T> f;
            load_m(f.m, mats, k);
            dispatch_elem<T>(st, k, f);
        } else if (cls == D1_RX) {
            FDense1RX<T> f;
            load_m(f.m, mats, k);
            dispatch_elem<T>(st, k, f);
        } else if (cls == D1_R0) {
            FDense1R0<T> f;
            load_m(f.m, mats, k);
            dispatch_elem<T>(st, k, f);
        } else {
            FDense1<T> f;
            load_m(f.m, mats, k);
            dispatch_elem<T>(st, k, f);
        }
        return;
    }
    case F_DIAG1: { FDiag1<T> f; load_m(f.d, mats, k); dispatch_elem<T>(st, k, f); return; }
    case F_PHASE: { FPhase<T> f; load_m(f.d, mats, k); dispatch_elem<T>(st, k, f); return; }
    case F_DIAG2: { FDiag2<T> f; load_m(f.d, mats, k); dispatch_elem<T>(st, k, f); return; }
    case F_DENSE2: { FDense2<T> f; load_m(f.m, mats, k); dispatch_elem<T>(st, k, f); return; }
    case F_DIAGK: {
        std::vector<T> tab(k.nmat);
        load_m(tab.data(), mats, k);
        const T *dtab = (const T *)upload_params(st, tab.data(), tab.size() * sizeof(T));
        const int4 qa = make_int4(k.pos[0], k.pos[1], k.pos[2], k.pos[3]);
        const int4 qb = make_int4(k.pos[4], k.pos[5], k.pos[6], k.pos[7]);
        if constexpr (std::is_same<T, double>::value) {
            auto kern = k_diag_general<double, 1>;
            const uint64_t ne = 1ull << n;
            const int grid = persistent_grid((const void *)kern, kThreads, 0, (ne + kThreads - 1) / kThreads);
            kern<<<grid, kThreads, 0, st.stream>>>((double2 *)st.psi, ne, k.k, qa, qb, dtab);
        } else {
            auto kern = k_diag_general<float, 2>;
            const uint64_t ne = 1ull << (n - 1);
            const int grid = persistent_grid((const void *)kern, kThreads, 0, (ne + kThreads - 1) / kThreads);
            kern<<<grid, kThreads, 0, st.stream>>>((float4 *)st.psi, ne, k.k, qa, qb, dtab);
        }
        QS_CUDA(cudaGetLastError());
        count_launch();
        return;
    }
    case F_DENSEK: {
        std::vector<T> tab(k.nmat);
        load_m(tab.data(), mats, k);
        const T *dm = (const T *)upload_params(st, tab.data(), tab.size() * sizeof(T));
        const int4 qa = make_int4(k.pos[0], k.pos[1], k.pos[2], k.pos[3]);
        const int4 qb = make_int4(k.pos[4], k.pos[5], k.pos[6], k.pos[7]);
        const uint64_t ng = 1ull << (n - k.k);
        using V = typename VecT<T, 1>::type;
        auto go = [&](auto kern) {
            const int grid = persistent_grid((const void *)kern, 128, 0, (ng + 127) / 128);
            kern<<<grid, 128, 0, st.stream>>>((V *)st.psi, ng, qa, qb, dm);
        };
        switch (k.k) {
        case 3: go(k_dense_general<T, 3>); break;
        case 4: go(k_dense_general<T, 4>); break;
        case 5: go(k_dense_general<T, 5>); break;
        case 6: go(k_dense_general<T, 6>); break;
        default: fail(QS_ERR_UNSUPPORTED, "dense block wider than 6 qubits");
        }
        QS_CUDA(cudaGetLastError());
        count_launch();
        return;
    }
    }
    fail(QS_ERR_INVALID, "unknown kernel op kind");
}

}  // namespace

static thread_local int t_yield_iters = 0;

LaunchYield::LaunchYield(int iters) : prev(t_yield_iters) { t_yield_iters = iters; }
LaunchYield::~LaunchYield() { t_yield_iters = prev; }

// Persistent grid size: SMs x resident blocks of this kernel (cached per kernel).
int persistent_grid(const void *fn, int threads, size_t smem, uint64_t work_blocks) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, size_t>, int> occ;
    int per_sm;
    {
        std::lock_guard<std::mutex> lk(mu);
        const auto key = std::make_tuple(fn, threads, smem);
        auto it = occ.find(key);
        if (it == occ.end()) {
            int b = 0;
            QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem));
            it = occ.emplace(key, std::max(b, 1)).first;
        }
        per_sm = it->second;
    }
    uint64_t full = (uint64_t)device_sm_count() * per_sm;
    if (t_yield_iters > 0)
        full = std::max<uint64_t>(full, std::min<uint64_t>((work_blocks + t_yield_iters - 1) / t_yield_iters,
                                                           (uint64_t)INT32_MAX));
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(full, work_blocks));
}

void launch_stream_op(DeviceState &st, const Op &op) {
    if (op.kind == K_PHASEFN) {
        launch_phasefn(st, op);
        return;
    }
    if (st.dtype == QS_C128) launch_typed<double>(st, op);
    else launch_typed<float>(st, op);
}

}  // namespace qs
