// K1: streaming gate kernels — one gate, one pass over the state vector.
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
#include <unordered_map>

#include "qs_internal.h"

namespace qs {
namespace {

template <typename T, int L> struct VecT;
template <> struct VecT<double, 1> { using type = double2; };
template <> struct VecT<float, 1> { using type = float2; };
template <> struct VecT<float, 2> { using type = float4; };

template <typename T, int L> struct Amp { T r[L], i[L]; };

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
__device__ __forceinline__ void stv(double2 *p, const Amp<double, 1> &a) {
    *p = make_double2(a.r[0], a.i[0]);
}
__device__ __forceinline__ void stv(float2 *p, const Amp<float, 1> &a) {
    *p = make_float2(a.r[0], a.i[0]);
}
__device__ __forceinline__ void stv(float4 *p, const Amp<float, 2> &a) {
    *p = make_float4(a.r[0], a.i[0], a.r[1], a.i[1]);
}

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

// ---- functors: each transforms the NT touched elements of one group --------------
template <typename T> struct FH {  // (a+b, a-b)/sqrt2
    static constexpr int NT = 2;
    T r;
    template <int L> __device__ void operator()(Amp<T, L> *v) const {
#pragma unroll
        for (int l = 0; l < L; l++) {
            const T ar = v[0].r[l], ai = v[0].i[l], br = v[1].r[l], bi = v[1].i[l];
            v[0].r[l] = (ar + br) * r; v[0].i[l] = (ai + bi) * r;
            v[1].r[l] = (ar - br) * r; v[1].i[l] = (ai - bi) * r;
        }
    }
};
template <typename T> struct FSwap {  // X, CNOT on the control=1 half, SWAP on 01/10
    static constexpr int NT = 2;
    template <int L> __device__ void operator()(Amp<T, L> *v) const {
        const Amp<T, L> t = v[0];
        v[0] = v[1];
        v[1] = t;
    }
};
template <typename T> struct FDense1 {  // 2x2 complex matrix
    static constexpr int NT = 2;
    T m[8];  // m00 m01 m10 m11 as (re, im)
    template <int L> __device__ void operator()(Amp<T, L> *v) const {
#pragma unroll
        for (int l = 0; l < L; l++) {
            const T ar = v[0].r[l], ai = v[0].i[l], br = v[1].r[l], bi = v[1].i[l];
            cdot2(v[0].r[l], v[0].i[l], m[0], m[1], ar, ai, m[2], m[3], br, bi);
            cdot2(v[1].r[l], v[1].i[l], m[4], m[5], ar, ai, m[6], m[7], br, bi);
        }
    }
};
template <typename T> struct FDiag1 {  // diag(d0, d1)
    static constexpr int NT = 2;
    T d[4];
    template <int L> __device__ void operator()(Amp<T, L> *v) const {
#pragma unroll
        for (int t = 0; t < 2; t++)
#pragma unroll
            for (int l = 0; l < L; l++) {
                const T xr = v[t].r[l], xi = v[t].i[l];
                v[t].r[l] = fma(d[2 * t], xr, -d[2 * t + 1] * xi);
                v[t].i[l] = fma(d[2 * t], xi, d[2 * t + 1] * xr);
            }
    }
};
template <typename T> struct FPhase {  // one touched element times e^{i a}
    static constexpr int NT = 1;
    T c, s;
    template <int L> __device__ void operator()(Amp<T, L> *v) const {
#pragma unroll
        for (int l = 0; l < L; l++) {
            const T xr = v[0].r[l], xi = v[0].i[l];
            v[0].r[l] = fma(c, xr, -s * xi);
            v[0].i[l] = fma(c, xi, s * xr);
        }
    }
};
template <typename T> struct FNeg {  // one touched element times -1 (Z, CZ)
    static constexpr int NT = 1;
    template <int L> __device__ void operator()(Amp<T, L> *v) const {
#pragma unroll
        for (int l = 0; l < L; l++) {
            v[0].r[l] = -v[0].r[l];
            v[0].i[l] = -v[0].i[l];
        }
    }
};
template <typename T> struct FDiag2 {  // four phases (RZZ and other 2-qubit diagonals)
    static constexpr int NT = 4;
    T d[8];
    template <int L> __device__ void operator()(Amp<T, L> *v) const {
#pragma unroll
        for (int t = 0; t < 4; t++)
#pragma unroll
            for (int l = 0; l < L; l++) {
                const T xr = v[t].r[l], xi = v[t].i[l];
                v[t].r[l] = fma(d[2 * t], xr, -d[2 * t + 1] * xi);
                v[t].i[l] = fma(d[2 * t], xi, d[2 * t + 1] * xr);
            }
    }
};
template <typename T> struct FDense2 {  // 4x4 complex matrix
    static constexpr int NT = 4;
    T m[32];
    template <int L> __device__ void operator()(Amp<T, L> *v) const {
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
};

constexpr int kThreads = 256;

// Inserts a zero bit at each of the NF sorted positions fb[] of x.
template <int NF>
__device__ __forceinline__ uint64_t insert_zeros(uint64_t x, const StreamGeom &g) {
#pragma unroll
    for (int j = 0; j < NF; j++) {
        const int b = g.fb[j];
        x = ((x >> b) << (b + 1)) | (x & ((1ull << b) - 1ull));
    }
    return x;
}

template <typename T, int L, int NF, int U, typename F>
__global__ void __launch_bounds__(kThreads)
k_stream(typename VecT<T, L>::type *__restrict__ psi, const StreamGeom g, const F f) {
    constexpr int NT = F::NT;
    const uint64_t per_iter = (uint64_t)kThreads * U;
    for (uint64_t b0 = (uint64_t)blockIdx.x * per_iter; b0 < g.n_groups;
         b0 += (uint64_t)gridDim.x * per_iter) {
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
            if (b0 + (uint64_t)u * kThreads + threadIdx.x < g.n_groups) f(v[u]);
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
k_diag_general(typename VecT<T, L>::type *__restrict__ psi, uint64_t n_elem, int k, int4 qa,
               int4 qb, const T *__restrict__ d) {
    const int qs_[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
    for (uint64_t e = (uint64_t)blockIdx.x * kThreads + threadIdx.x; e < n_elem;
         e += (uint64_t)gridDim.x * kThreads) {
        Amp<T, L> a;
        ldv(psi + e, a);
#pragma unroll
        for (int l = 0; l < L; l++) {
            const uint64_t x = e * L + l;
            uint32_t s = 0;
            for (int j = 0; j < k; j++) s |= (uint32_t)((x >> qs_[j]) & 1ull) << (k - 1 - j);
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
    const int q[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
    int sorted[K];
#pragma unroll
    for (int j = 0; j < K; j++) sorted[j] = q[j];
    for (int a = 1; a < K; a++)  // insertion sort of the operand bits (tiny)
        for (int b = a; b > 0 && sorted[b - 1] > sorted[b]; b--) {
            const int t = sorted[b]; sorted[b] = sorted[b - 1]; sorted[b - 1] = t;
        }
    uint64_t off[D];
#pragma unroll
    for (int s = 0; s < D; s++) {
        uint64_t o = 0;
#pragma unroll
        for (int j = 0; j < K; j++) o |= (uint64_t)((s >> (K - 1 - j)) & 1) << q[j];
        off[s] = o;
    }
    for (uint64_t gi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < n_groups;
         gi += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x = gi;
#pragma unroll
        for (int j = 0; j < K; j++) {
            const int b = sorted[j];
            x = ((x >> b) << (b + 1)) | (x & ((1ull << b) - 1ull));
        }
        T vr[D], vi[D];
#pragma unroll
        for (int s = 0; s < D; s++) {
            Amp<T, 1> a;
            ldv(psi + x + off[s], a);
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
            stv(psi + x + off[r], o);
        }
    }
}

// Persistent grid size: SMs x resident blocks of this kernel (cached per kernel).
int grid_for(const void *fn, int threads, size_t smem, uint64_t work_blocks) {
    static std::mutex mu;
    static std::unordered_map<const void *, int> occ;
    int per_sm;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = occ.find(fn);
        if (it == occ.end()) {
            int b = 0;
            QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem));
            it = occ.emplace(fn, std::max(b, 1)).first;
        }
        per_sm = it->second;
    }
    const uint64_t full = (uint64_t)device_sm_count() * per_sm;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(full, work_blocks));
}

template <typename T, int L, int NF, typename F>
void run(DeviceState &st, const StreamGeom &g, const F &f) {
    constexpr int NT = F::NT;
    constexpr int U = NT == 4 ? 2 : (NT == 2 ? 4 : 8);
    auto kern = k_stream<T, L, NF, U, F>;
    const uint64_t per_iter = (uint64_t)kThreads * U;
    const int grid = grid_for((const void *)kern, kThreads, 0, (g.n_groups + per_iter - 1) / per_iter);
    kern<<<grid, kThreads, 0, st.stream>>>((typename VecT<T, L>::type *)st.psi, g, f);
    QS_CUDA(cudaGetLastError());
    count_launch();
}

template <typename T, int L, typename F>
void run_nf(DeviceState &st, const StreamGeom &g, const F &f) {
    if (g.nf == 1) run<T, L, 1>(st, g, f);
    else if (g.nf == 2) run<T, L, 2>(st, g, f);
    else fail(QS_ERR_INVALID, "streaming op with unsupported fixed-bit count");
}

// Element geometry from amplitude geometry: float4 elements (two amplitudes) when the
// dtype is complex64 and no fixed bit is bit 0.
template <typename T, typename F>
void dispatch_elem(DeviceState &st, StreamGeom g, const F &f) {
    if constexpr (std::is_same<T, double>::value) {
        run_nf<T, 1>(st, g, f);
        return;
    } else if (g.fb[0] >= 1) {
        for (int j = 0; j < g.nf; j++) g.fb[j] -= 1;
        g.set_mask >>= 1;
        for (int t = 0; t < g.nt; t++) g.off[t] >>= 1;
        g.n_groups >>= 1;
        run_nf<float, 2>(st, g, f);
    } else {
        run_nf<float, 1>(st, g, f);
    }
}

bool is_one(cd z) { return z == cd(1.0, 0.0); }
bool is_minus_one(cd z) { return z == cd(-1.0, 0.0); }

StreamGeom geom(int n, std::initializer_list<int> fixed, uint64_t set_mask,
                std::initializer_list<uint64_t> offs) {
    StreamGeom g{};
    g.nf = 0;
    for (int b : fixed) g.fb[g.nf++] = b;
    std::sort(g.fb, g.fb + g.nf);
    g.set_mask = set_mask;
    g.nt = 0;
    for (uint64_t o : offs) g.off[g.nt++] = o;
    g.n_groups = 1ull << (n - g.nf);
    return g;
}

template <typename T>
void set_m(T *dst, const std::vector<cd> &m) {
    for (size_t i = 0; i < m.size(); i++) {
        dst[2 * i] = (T)m[i].real();
        dst[2 * i + 1] = (T)m[i].imag();
    }
}

template <typename T>
void launch_typed(DeviceState &st, const Op &op) {
    const int n = st.n;
    switch (op.kind) {
    case K_H: {
        FH<T> f;
        f.r = (T)(1.0 / std::sqrt(2.0));
        dispatch_elem<T>(st, geom(n, {op.q[0]}, 0, {0, 1ull << op.q[0]}), f);
        return;
    }
    case K_PERM1:
        dispatch_elem<T>(st, geom(n, {op.q[0]}, 0, {0, 1ull << op.q[0]}), FSwap<T>{});
        return;
    case K_DIAG1: {
        const int q = op.q[0];
        if (is_one(op.m[0])) {
            const StreamGeom g = geom(n, {q}, 1ull << q, {0});
            if (is_minus_one(op.m[1])) {
                dispatch_elem<T>(st, g, FNeg<T>{});
            } else {
                FPhase<T> f;
                f.c = (T)op.m[1].real(); f.s = (T)op.m[1].imag();
                dispatch_elem<T>(st, g, f);
            }
        } else {
            FDiag1<T> f;
            set_m(f.d, op.m);
            dispatch_elem<T>(st, geom(n, {q}, 0, {0, 1ull << q}), f);
        }
        return;
    }
    case K_DENSE1: {
        FDense1<T> f;
        set_m(f.m, op.m);
        dispatch_elem<T>(st, geom(n, {op.q[0]}, 0, {0, 1ull << op.q[0]}), f);
        return;
    }
    case K_CTRL1: {
        const int c = op.q[0], t = op.q[1];
        const std::vector<cd> &u = op.m;
        const bool diag = u[1] == cd(0.0) && u[2] == cd(0.0);
        if (u[0] == cd(0.0) && u[3] == cd(0.0) && is_one(u[1]) && is_one(u[2])) {
            dispatch_elem<T>(st, geom(n, {c, t}, 1ull << c, {0, 1ull << t}), FSwap<T>{});
        } else if (diag && is_one(u[0])) {
            const StreamGeom g = geom(n, {c, t}, (1ull << c) | (1ull << t), {0});
            if (is_minus_one(u[3])) {
                dispatch_elem<T>(st, g, FNeg<T>{});
            } else {
                FPhase<T> f;
                f.c = (T)u[3].real(); f.s = (T)u[3].imag();
                dispatch_elem<T>(st, g, f);
            }
        } else if (diag) {
            FDiag1<T> f;
            set_m(f.d, {u[0], u[3]});
            dispatch_elem<T>(st, geom(n, {c, t}, 1ull << c, {0, 1ull << t}), f);
        } else {
            FDense1<T> f;
            set_m(f.m, u);
            dispatch_elem<T>(st, geom(n, {c, t}, 1ull << c, {0, 1ull << t}), f);
        }
        return;
    }
    case K_SWAP: {
        const int a = op.q[0], b = op.q[1];
        dispatch_elem<T>(st, geom(n, {a, b}, 0, {1ull << a, 1ull << b}), FSwap<T>{});
        return;
    }
    case K_DIAG: {
        if (op.k == 1) {
            Op o1 = op;
            o1.kind = K_DIAG1;
            launch_typed<T>(st, o1);
            return;
        }
        if (op.k == 2) {
            const int a = op.q[0], b = op.q[1];
            const uint64_t A = 1ull << a, B = 1ull << b;
            if (is_one(op.m[0]) && is_one(op.m[1]) && is_one(op.m[2])) {
                const StreamGeom g = geom(n, {a, b}, A | B, {0});
                if (is_minus_one(op.m[3])) {
                    dispatch_elem<T>(st, g, FNeg<T>{});
                } else {
                    FPhase<T> f;
                    f.c = (T)op.m[3].real(); f.s = (T)op.m[3].imag();
                    dispatch_elem<T>(st, g, f);
                }
            } else {
                FDiag2<T> f;
                set_m(f.d, op.m);
                dispatch_elem<T>(st, geom(n, {a, b}, 0, {0, B, A, A | B}), f);
            }
            return;
        }
        // general diagonal: table on the device
        std::vector<T> tab(2 * op.m.size());
        set_m(tab.data(), op.m);
        T *dtab = (T *)upload_params(st, tab.data(), tab.size() * sizeof(T));
        int qq[8] = {0};
        for (int j = 0; j < op.k; j++) qq[j] = op.q[j];
        const int4 qa = make_int4(qq[0], qq[1], qq[2], qq[3]), qb = make_int4(qq[4], qq[5], qq[6], qq[7]);
        if constexpr (std::is_same<T, double>::value) {
            auto kern = k_diag_general<double, 1>;
            const uint64_t ne = 1ull << n;
            const int grid = grid_for((const void *)kern, kThreads, 0, (ne + kThreads - 1) / kThreads);
            kern<<<grid, kThreads, 0, st.stream>>>((double2 *)st.psi, ne, op.k, qa, qb, (const double *)dtab);
        } else if (n >= 1) {
            auto kern = k_diag_general<float, 2>;
            const uint64_t ne = 1ull << (n - 1);
            const int grid = grid_for((const void *)kern, kThreads, 0, (ne + kThreads - 1) / kThreads);
            kern<<<grid, kThreads, 0, st.stream>>>((float4 *)st.psi, ne, op.k, qa, qb, (const float *)dtab);
        }
        QS_CUDA(cudaGetLastError());
        count_launch();
        return;
    }
    case K_DENSE: {
        if (op.k == 2) {
            FDense2<T> f;
            set_m(f.m, op.m);
            const uint64_t A = 1ull << op.q[0], B = 1ull << op.q[1];
            dispatch_elem<T>(st, geom(n, {op.q[0], op.q[1]}, 0, {0, B, A, A | B}), f);
            return;
        }
        std::vector<T> tab(2 * op.m.size());
        set_m(tab.data(), op.m);
        T *dm = (T *)upload_params(st, tab.data(), tab.size() * sizeof(T));
        int qq[8] = {0};
        for (int j = 0; j < op.k; j++) qq[j] = op.q[j];
        const int4 qa = make_int4(qq[0], qq[1], qq[2], qq[3]), qb = make_int4(qq[4], qq[5], qq[6], qq[7]);
        const uint64_t ng = 1ull << (n - op.k);
        using V = typename VecT<T, 1>::type;
        auto go = [&](auto kern) {
            const int grid = grid_for((const void *)kern, 128, 0, (ng + 127) / 128);
            kern<<<grid, 128, 0, st.stream>>>((V *)st.psi, ng, qa, qb, (const T *)dm);
        };
        switch (op.k) {
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
    fail(QS_ERR_INVALID, "unknown op kind");
}

}  // namespace

void launch_stream_op(DeviceState &st, const Op &op) {
    if (st.dtype == QS_C128) launch_typed<double>(st, op);
    else launch_typed<float>(st, op);
}

double stream_bytes(const Op &op, int n, int dtype) {
    const double B = dtype == QS_C128 ? 16.0 : 8.0;
    const double full = 2.0 * B * (double)(1ull << n);   // read + write of every amplitude
    // sub-sector selection (bit below the 32-byte sector) touches every sector anyway
    const int sector_bits = dtype == QS_C128 ? 1 : 2;
    auto frac_ok = [&](int q) { return q >= sector_bits; };
    switch (op.kind) {
    case K_CTRL1: {
        const cd *u = op.m.data();
        const bool phase = u[1] == cd(0.0) && u[2] == cd(0.0) && u[0] == cd(1.0);
        if (phase) return (frac_ok(op.q[0]) && frac_ok(op.q[1])) ? full / 4 : (frac_ok(op.q[0]) || frac_ok(op.q[1]) ? full / 2 : full);
        return frac_ok(op.q[0]) ? full / 2 : full;
    }
    case K_SWAP:
        return (frac_ok(op.q[0]) && frac_ok(op.q[1])) ? full / 2 : full;
    case K_DIAG1:
        return (op.m[0] == cd(1.0) && frac_ok(op.q[0])) ? full / 2 : full;
    case K_DIAG:
        if (op.k == 2 && op.m[0] == cd(1.0) && op.m[1] == cd(1.0) && op.m[2] == cd(1.0)) {
            const int f = (int)frac_ok(op.q[0]) + (int)frac_ok(op.q[1]);
            return f == 2 ? full / 4 : (f == 1 ? full / 2 : full);
        }
        return full;
    default:
        return full;
    }
}

}  // namespace qs
