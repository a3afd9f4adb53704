// K4/K5: reductions and simple state kernels.
//
//  * norm and <Z_q> for every q in one read pass.  <Z_q> = sum_x |a_x|^2 (1 - 2 bit_q(x))
//    = total - 2 S_q with S_q the probability mass on bit_q = 1.  Three levels: a block
//    of the first level owns a contiguous chunk of 2^cb amplitudes, so every qubit >= cb
//    is constant over it and only its total is needed for that qubit (qubits < cb are
//    split into thread bits and loop bits); the second level combines groups of 256 such
//    records, adding the 8 qubits spelled by the record index within the group; the last
//    level combines the few second-level records.  Everything is summed in a fixed order
//    (per-thread pairwise trees, fixed butterfly trees, fixed upper levels), so results
//    are bitwise reproducible whatever else runs on the GPU.  complex128 sums in FP64;
//    complex64 sums each thread's groups of 16 exact squares in double-float FP32 and
//    everything above in FP64 (FP64 throughput is the limit of these passes on GB300).
//  * top-K |a|^2: exact radix select of the K-th largest key (the bit pattern of the
//    non-negative probability, monotone in its value), then a deterministic gather of
//    the elements above it and of the lowest-index ties, then one-block bitonic sort.
//  * |0...0> and scaling.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "capi_util.h"
#include "qs_internal.h"

namespace qs {
namespace {

__device__ __forceinline__ double prob(double2 a) {
    return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
}
__device__ __forceinline__ double prob(float2 a) {
    // products of floats are exact in double
    return __dadd_rn(__dmul_rn((double)a.x, (double)a.x), __dmul_rn((double)a.y, (double)a.y));
}
// Exact float -> double by integer bit operations (the hardware conversion runs on the
// FP64 pipe); zero, subnormal and non-finite values take the hardware conversion.
__device__ __forceinline__ double f2d_exact(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return (double)x;
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)((b & 7u) << 29));
}
// Sums of |a|^2 inside one thread of the first level, over a group of 16 or 32 amplitudes.
// complex128: FP64, with a pair of amplitudes summed as one chain of fused multiply-adds.
// complex64: the squares of the stored floats are exact as FP32 pairs (x*x and
// fma(x, x, -x*x)) and are added as double-float values (hi, lo: an FP32 two-sum per
// addition, then a renormalisation), so a group's sums run on the FP32 pipe and the FP64
// pipe sees one exact conversion and one addition per group sum.  Each double-float
// addition of non-negative terms errs by at most 3 * 2^-48 of its result and a leaf (one
// |a|^2) by the same, so a pairwise tree of depth <= 5 is within 18 * 2^-48 (6.4e-14) of
// its exact sum.
struct SumF64 {
    using T = double;
    static __device__ __forceinline__ T add(T a, T b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ T leaf(double2 a) { return __fma_rn(a.x, a.x, __dmul_rn(a.y, a.y)); }
    // |a|^2 + |b|^2 with pb = |b|^2: four FP64 instructions for two amplitudes
    static __device__ __forceinline__ T pair(double2 a, double2 b, T &pb) {
        pb = leaf(b);
        return __fma_rn(a.x, a.x, __fma_rn(a.y, a.y, pb));
    }
    static __device__ __forceinline__ double to_double(T a) { return a; }
};
struct SumDF32 {
    using T = float2;  // (hi, lo), |lo| <= ulp(hi) / 2
    // hi + lo of s + l rounded to nearest, exactly (Fast2Sum: |s| >= |l| here)
    static __device__ __forceinline__ T renorm(float s, float l) {
        const float h = __fadd_rn(s, l);
        return make_float2(h, __fsub_rn(l, __fsub_rn(h, s)));
    }
    static __device__ __forceinline__ T add(T a, T b) {
        const float s = __fadd_rn(a.x, b.x);
        const float bb = __fsub_rn(s, a.x);
        const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));  // TwoSum
        return renorm(s, __fadd_rn(__fadd_rn(a.y, b.y), e));
    }
    static __device__ __forceinline__ T leaf(float2 a) {
        const float hx = __fmul_rn(a.x, a.x), hy = __fmul_rn(a.y, a.y);
        const float lx = __fmaf_rn(a.x, a.x, -hx), ly = __fmaf_rn(a.y, a.y, -hy);
        const float s = __fadd_rn(hx, hy);
        const float bb = __fsub_rn(s, hx);
        const float e = __fadd_rn(__fsub_rn(hx, __fsub_rn(s, bb)), __fsub_rn(hy, bb));
        return renorm(s, __fadd_rn(__fadd_rn(lx, ly), e));
    }
    static __device__ __forceinline__ T pair(float2 a, float2 b, T &pb) {
        pb = leaf(b);
        return add(leaf(a), pb);
    }
    // hi + lo spans at most 48 significant bits: the FP64 sum is exact
    static __device__ __forceinline__ double to_double(T a) { return __dadd_rn(f2d_exact(a.x), f2d_exact(a.y)); }
};
template <typename V> struct SumOf;
template <> struct SumOf<double2> { using S = SumF64; };
template <> struct SumOf<float2> { using S = SumDF32; };


// Butterfly sum over a warp: fixed order, identical result in every lane.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Pairwise sum of x[0..N-1] (N a power of two) in a fixed order.
template <typename S, int N, typename A>
__device__ __forceinline__ A tree_sum(const A *x) {
    if constexpr (N == 1) return x[0];
    else return S::add(tree_sum<S, N / 2>(x), tree_sum<S, N / 2>(x + N / 2));
}

// Levels L.. of a group's tree, M nodes at level L in cur[]: mass[L] = sum of the odd
// nodes (bit L of the loop index set), then the pair sums move up; returns the group total.
template <typename S, int L, int M, int BITS>
struct TreeLevels {
    using A = typename S::T;
    static __device__ __forceinline__ A run(A *cur, A *mass) {
        if constexpr (M == 1) {
            return cur[0];
        } else {
            if (BITS) {
                A odd[M / 2];
#pragma unroll
                for (int i = 0; i < M / 2; i++) odd[i] = cur[2 * i + 1];
                mass[L] = tree_sum<S, M / 2>(odd);
            }
#pragma unroll
            for (int i = 0; i < M / 2; i++) cur[i] = S::add(cur[2 * i], cur[2 * i + 1]);
            return TreeLevels<S, L + 1, M / 2, BITS>::run(cur, mass);
        }
    }
};

// Level 1: part[blk*(cb+1) + 0] = block total; part[blk*(cb+1) + 1 + q] = mass with bit q
// set, q < cb.  JB = loop bits per thread (cb = tb + JB); BITS = 0: totals only (the same
// operations in the same order, so a norm equals the total of a <Z_q> call bit for bit).
// A thread loads its amplitudes in groups of 2^U (the low U loop bits; U = 4 for
// complex128, 5 for complex64) and sums each group by a fixed pairwise tree; the mass of
// low loop bit l is a pairwise sum of the odd nodes of the tree's level l; the high loop
// bits take the group totals.  Group results go to FP64 accumulators, so no double-float
// sum spans more than one tree of depth <= 5.
template <typename V, int JB, int BITS>
__global__ void __launch_bounds__(256)
k_expz_part(const V *__restrict__ psi, int cb, int tb, double *__restrict__ part) {
    using S = typename SumOf<V>::S;
    using A = typename S::T;
    constexpr int UMAX = std::is_same<V, float2>::value ? 5 : 4;
    constexpr int U = JB < UMAX ? JB : UMAX;
    constexpr int NJ = JB > 0 ? JB : 1;
    constexpr int H = U > 0 ? (1 << (U - 1)) : 1;  // pairs per group
    __shared__ double s_tot[256];
    __shared__ double s_j[NJ][256];
    const int T = 1 << tb, t = threadIdx.x;
    const uint64_t start = (uint64_t)blockIdx.x << cb;
    double tot = 0.0, jacc[NJ];
#pragma unroll
    for (int b = 0; b < NJ; b++) jacc[b] = 0.0;
#pragma unroll 1
    for (int g = 0; g < (1 << (JB - U)); g++) {
        V v[1 << U];
#pragma unroll
        for (int j = 0; j < (1 << U); j++) v[j] = psi[start + ((uint64_t)((g << U) + j) << tb) + t];
        A gt, mass[U > 0 ? U : 1];
        if constexpr (U == 0) {
            gt = S::leaf(v[0]);
        } else {
            A cur[H], odd[H];
#pragma unroll
            for (int i = 0; i < H; i++) cur[i] = S::pair(v[2 * i], v[2 * i + 1], odd[i]);
            if (BITS) mass[0] = tree_sum<S, H>(odd);
            gt = TreeLevels<S, 1, H, BITS>::run(cur, mass);
        }
        const double gd = S::to_double(gt);
        tot = __dadd_rn(tot, gd);
        if (BITS) {
#pragma unroll
            for (int l = 0; l < U; l++) jacc[l] = __dadd_rn(jacc[l], S::to_double(mass[l]));
#pragma unroll
            for (int b = U; b < JB; b++)
                if ((g >> (b - U)) & 1) jacc[b] = __dadd_rn(jacc[b], gd);
        }
    }
    s_tot[t] = tot;
    if (BITS)
#pragma unroll
        for (int b = 0; b < JB; b++) s_j[b][t] = jacc[b];
    __syncthreads();
    const int n_out = BITS ? cb + 1 : 1;
    const int warp = t >> 5, lane = t & 31, nw = (T + 31) >> 5;
    for (int r = warp; r < n_out; r += nw) {
        auto val = [&](int u) -> double {
            if (r == 0) return s_tot[u];
            if (r - 1 < tb) return ((u >> (r - 1)) & 1) ? s_tot[u] : 0.0;
            return s_j[r - 1 - tb][u];
        };
        double v = 0.0;
        if (T >= 32) {
            for (int u = lane; u < T; u += 32) v += val(u);
            v = warp_sum(v);
        } else if (lane == 0) {  // tiny blocks: lane 0 adds the T lanes in order
            for (int u = 0; u < T; u++) v += val(u);
        }
        if (lane == 0) part[(uint64_t)blockIdx.x * (cb + 1) + r] = v;
    }
}

// Level 2: one block per group of G = 2^gb consecutive level-1 records (G <= 256): record
// layout [total, S_0 .. S_{cb-1}, S_cb .. S_{cb+gb-1}] (r2 = cb + 1 + gb doubles); the
// last gb masses come from the totals of the records whose index in the group has that
// bit set.  Each warp owns outputs; lane l adds records l, l + 32, ... in order, then a
// fixed butterfly.
__global__ void __launch_bounds__(256)
k_expz_mid(const double *__restrict__ part, int cb, int gb, int bits, double *__restrict__ mid) {
    const int G = 1 << gb, r1 = cb + 1, r2 = bits ? cb + 1 + gb : 1;
    const uint64_t g0 = (uint64_t)blockIdx.x << gb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int o = warp; o < r2; o += 8) {
        double v = 0.0;
        for (int u = lane; u < G; u += 32) {
            const double *rec = part + (g0 + (uint64_t)u) * r1;
            if (o < r1) v += rec[o];
            else if ((u >> (o - r1)) & 1) v += rec[0];
        }
        v = warp_sum(v);
        if (lane == 0) mid[(uint64_t)blockIdx.x * r2 + o] = v;
    }
}

// Level 3: out[0] = total, out[1 + q] = <Z_q> for q < n.  One block per output, over the
// nmid level-2 records (record width r2 = cb + 1 + gb; qubits >= cb + gb from totals).
__global__ void __launch_bounds__(256)
k_expz_final(const double *__restrict__ mid, uint64_t nmid, int qlo, int r2, double *__restrict__ out) {
    __shared__ double s[256];
    const int o = blockIdx.x;  // 0: total, 1+q: qubit q
    const int q = o - 1;
    double tot = 0.0, v = 0.0;
    for (uint64_t b = threadIdx.x; b < nmid; b += 256) {
        const double bt = mid[b * r2];
        tot += bt;
        if (q >= 0) {
            if (q < qlo) v += mid[b * r2 + 1 + q];
            else if ((b >> (q - qlo)) & 1) v += bt;
        }
    }
    // fixed-order tree over the 256 partials
    for (int pass = 0; pass < 2; pass++) {
        s[threadIdx.x] = pass == 0 ? tot : v;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
            __syncthreads();
        }
        if (pass == 0) tot = s[0];
        else v = s[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[o] = (q < 0) ? tot : tot - 2.0 * v;
}

template <typename V, int JB>
void part_launch(const void *psi, uint64_t nblk, int cb, int tb, bool bits, double *part, cudaStream_t st) {
    if (bits) k_expz_part<V, JB, 1><<<(unsigned)nblk, 1 << tb, 0, st>>>((const V *)psi, cb, tb, part);
    else k_expz_part<V, JB, 0><<<(unsigned)nblk, 1 << tb, 0, st>>>((const V *)psi, cb, tb, part);
}

template <typename V>
void part_dispatch(const void *psi, uint64_t nblk, int cb, int tb, bool bits, double *part, cudaStream_t st) {
    switch (cb - tb) {
    case 0: part_launch<V, 0>(psi, nblk, cb, tb, bits, part, st); break;
    case 1: part_launch<V, 1>(psi, nblk, cb, tb, bits, part, st); break;
    case 2: part_launch<V, 2>(psi, nblk, cb, tb, bits, part, st); break;
    case 3: part_launch<V, 3>(psi, nblk, cb, tb, bits, part, st); break;
    case 4: part_launch<V, 4>(psi, nblk, cb, tb, bits, part, st); break;
    case 5: part_launch<V, 5>(psi, nblk, cb, tb, bits, part, st); break;
    case 6: part_launch<V, 6>(psi, nblk, cb, tb, bits, part, st); break;
    case 7: part_launch<V, 7>(psi, nblk, cb, tb, bits, part, st); break;
    case 8: part_launch<V, 8>(psi, nblk, cb, tb, bits, part, st); break;
    case 9: part_launch<V, 9>(psi, nblk, cb, tb, bits, part, st); break;
    case 10: part_launch<V, 10>(psi, nblk, cb, tb, bits, part, st); break;
    default: fail(QS_ERR_INVALID, "reduction block too large");
    }
}

// Scratch doubles of the three-level pipeline for n qubits, first-level blocks of 2^cb.
size_t expz_pipeline_doubles(int n, int cb) {
    const uint64_t nblk = 1ull << (n - cb);
    const int gb = (int)std::min<uint64_t>(8, (uint64_t)(n - cb));
    const uint64_t nmid = nblk >> gb;
    return nblk * (cb + 1) + nmid * (cb + 1 + gb) + n + 1;
}

// Norm (and <Z_q> if bits) of the state at psi into out (n + 1 doubles, device); scratch
// holds expz_pipeline_doubles(n, cb) doubles (out may be its tail).
void expz_pipeline(const void *psi, bool c128, int n, int cb, bool bits, double *scratch, double *out,
                   cudaStream_t st) {
    const int tb = std::min(cb, 8);
    const uint64_t nblk = 1ull << (n - cb);
    const int gb = (int)std::min<uint64_t>(8, (uint64_t)(n - cb));
    const uint64_t nmid = nblk >> gb;
    double *part = scratch;
    double *mid = part + nblk * (cb + 1);
    if (c128) part_dispatch<double2>(psi, nblk, cb, tb, bits, part, st);
    else part_dispatch<float2>(psi, nblk, cb, tb, bits, part, st);
    QS_CUDA(cudaGetLastError());
    k_expz_mid<<<(unsigned)nmid, 256, 0, st>>>(part, cb, gb, bits ? 1 : 0, mid);
    QS_CUDA(cudaGetLastError());
    const int r2 = bits ? cb + 1 + gb : 1;
    k_expz_final<<<bits ? n + 1 : 1, 256, 0, st>>>(mid, nmid, cb + gb, r2, out);
    QS_CUDA(cudaGetLastError());
    count_launch(3);
}

__global__ void k_set_one(void *psi, int is_c128) {
    if (is_c128) ((double2 *)psi)[0] = make_double2(1.0, 0.0);
    else ((float2 *)psi)[0] = make_float2(1.0f, 0.0f);
}

// psi *= sqrt(norms[0] / norms[1]) (both squared norms in device memory, FP64)
template <typename V>
__global__ void __launch_bounds__(256) k_scale_ratio(V *__restrict__ psi, uint64_t n, const double *__restrict__ norms) {
    const double a = norms[0], b = norms[1];
    if (!(a > 0.0) || !(b > 0.0)) return;
    const double f = sqrt(a / b);
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (uint64_t)gridDim.x * 256) {
        V v = psi[i];
        v.x = (decltype(v.x))((double)v.x * f);
        v.y = (decltype(v.y))((double)v.y * f);
        psi[i] = v;
    }
}

template <typename V, typename S>
__global__ void __launch_bounds__(256) k_scale(V *__restrict__ psi, uint64_t n, S f) {
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (uint64_t)gridDim.x * 256) {
        V a = psi[i];
        a.x *= f;
        a.y *= f;
        psi[i] = a;
    }
}

// ---------------------------------------------------------------------------------
// Top-K.
struct SelState {
    unsigned long long prefix;  // key bits decided so far (high bits)
    unsigned long long need;    // how many elements with key matching prefix are still needed
    int shift;                  // bit position of the next digit's low end (for the last pass, 0)
    int pad;
};

__device__ __forceinline__ unsigned long long key_of(double2 a) {
    return (unsigned long long)__double_as_longlong(prob(a));
}
__device__ __forceinline__ unsigned long long key_of(float2 a) {
    return (unsigned long long)__double_as_longlong(prob(a));
}

constexpr int kDigitBits = 11;
constexpr int kBins = 1 << kDigitBits;

// Histogram of the next digit of keys whose bits above `hi_shift` equal prefix.
template <typename V>
__global__ void __launch_bounds__(256)
k_sel_hist(const V *__restrict__ psi, uint64_t n, const SelState *__restrict__ st, int hi_shift,
           int shift, unsigned long long *__restrict__ hist, const int *__restrict__ skip) {
    if (*skip) return;
    __shared__ unsigned int h[kBins];
    for (int i = threadIdx.x; i < kBins; i += 256) h[i] = 0;
    __syncthreads();
    const unsigned long long prefix = st->prefix;
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (uint64_t)gridDim.x * 256) {
        const unsigned long long k = key_of(psi[i]);
        const bool match = hi_shift >= 64 || (k >> hi_shift) == (prefix >> hi_shift);
        if (match) atomicAdd(&h[(k >> shift) & (kBins - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += 256)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

__global__ void k_sel_init(SelState *st, unsigned long long K, const int *skip) {
    if (*skip) return;
    st->prefix = 0ull;
    st->need = K;
    st->shift = 0;
    st->pad = 0;
}

// Picks the digit holding the need-th largest key among the matching ones.
__global__ void k_sel_pick(SelState *st, unsigned long long *hist, int shift, const int *skip) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || *skip) return;
    unsigned long long need = st->need, acc = 0;
    int d = kBins - 1;
    for (; d > 0; d--) {
        if (acc + hist[d] >= need) break;
        acc += hist[d];
    }
    st->prefix |= (unsigned long long)d << shift;
    st->need = need - acc;
    for (int i = 0; i < kBins; i++) hist[i] = 0;
}

// Per block of 2^cb consecutive indices: number of keys equal to the threshold.
template <typename V>
__global__ void __launch_bounds__(256)
k_tie_count(const V *__restrict__ psi, int cb, const SelState *__restrict__ st,
            unsigned int *__restrict__ cnt, const int *__restrict__ skip) {
    if (*skip) return;
    __shared__ unsigned int c;
    if (threadIdx.x == 0) c = 0;
    __syncthreads();
    const unsigned long long T = st->prefix;
    const uint64_t start = (uint64_t)blockIdx.x << cb;
    unsigned int mine = 0;
    for (uint64_t i = threadIdx.x; i < (1ull << cb); i += 256) mine += key_of(psi[start + i]) == T;
    atomicAdd(&c, mine);
    __syncthreads();
    if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

// Exclusive scan of the per-block tie counts (one block, fixed order).
__global__ void k_tie_scan(unsigned int *cnt, uint64_t nblk, const int *skip) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || *skip) return;
    unsigned long long acc = 0;
    for (uint64_t b = 0; b < nblk; b++) {
        const unsigned int c = cnt[b];
        cnt[b] = (unsigned int)std::min<unsigned long long>(acc, 0xffffffffull);
        acc += c;
    }
}

// Writes every key > T (slot by atomic counter: the order is fixed by the final sort) and
// the `need` lowest-index keys == T (slot by global tie rank, index order).
template <typename V>
__global__ void __launch_bounds__(256)
k_gather(const V *__restrict__ psi, int cb, const SelState *__restrict__ st, unsigned int K,
         const unsigned int *__restrict__ tie_base, unsigned int *__restrict__ gt_count,
         unsigned long long *__restrict__ out_key, unsigned long long *__restrict__ out_idx,
         const int *__restrict__ skip) {
    if (*skip) return;
    __shared__ unsigned int warp_cnt[8];
    __shared__ unsigned int running;
    const unsigned long long T = st->prefix, need = st->need;
    const unsigned int n_gt = K - (unsigned int)need;
    const uint64_t start = (uint64_t)blockIdx.x << cb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) running = tie_base[blockIdx.x];
    __syncthreads();
    for (uint64_t i0 = 0; i0 < (1ull << cb); i0 += 256) {
        const uint64_t x = start + i0 + threadIdx.x;
        const bool valid = i0 + threadIdx.x < (1ull << cb);
        const unsigned long long k = valid ? key_of(psi[x]) : 0ull;
        if (valid && k > T) {
            const unsigned int slot = atomicAdd(gt_count, 1u);
            if (slot < n_gt) { out_key[slot] = k; out_idx[slot] = x; }
        }
        const bool tie = valid && k == T;
        const unsigned int bal = __ballot_sync(0xffffffffu, tie);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        unsigned int before = running;
        for (int w = 0; w < warp; w++) before += warp_cnt[w];
        before += __popc(bal & ((1u << lane) - 1u));
        if (tie && before < need) {
            out_key[n_gt + before] = k;
            out_idx[n_gt + before] = x;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int tot = 0;
            for (int w = 0; w < 8; w++) tot += warp_cnt[w];
            running += tot;
        }
        __syncthreads();
    }
}

// One-block bitonic sort of P (power of two <= 4096) entries by (key desc, idx asc);
// entries beyond K are padding (key 0, idx max).  Writes idx and amplitudes (as doubles).
template <typename V>
__global__ void __launch_bounds__(1024)
k_topk_sort(const V *__restrict__ psi, const unsigned long long *key, const unsigned long long *idx, int K,
            int P, int n_in, const unsigned int *__restrict__ n_in_dev, unsigned long long *__restrict__ out_idx,
            double *__restrict__ out_amp, const int *__restrict__ skip, int skip_when) {
    // runs when *skip != skip_when: the exact pipeline's sort skips when the fast path ran,
    // the fast path's sort skips when it did not
    if ((*skip != 0) == (skip_when != 0)) return;
    extern __shared__ unsigned long long sm[];
    unsigned long long *sk = sm, *si = sm + P;
    if (n_in < 0) n_in = (int)min(*n_in_dev, (unsigned int)P);  // candidate count (fast path)
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        sk[i] = i < n_in ? key[i] : 0ull;
        si[i] = i < n_in ? idx[i] : ~0ull;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    // "before" = larger key, then smaller index
                    const bool i_before_j = sk[i] > sk[j] || (sk[i] == sk[j] && si[i] < si[j]);
                    const bool up = (i & size) == 0;  // this run sorted in "before" order
                    if (up ? !i_before_j : i_before_j) {
                        unsigned long long t = sk[i]; sk[i] = sk[j]; sk[j] = t;
                        t = si[i]; si[i] = si[j]; si[j] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        const unsigned long long x = si[i];
        out_idx[i] = x;
        const V a = psi[x];
        out_amp[2 * i] = (double)a.x;
        out_amp[2 * i + 1] = (double)a.y;
    }
}

// ---- top-K fast path: FP32 prefilter, exact FP64 keys for the candidates only ----------
// p32 = |a|^2 in FP32 from the amplitude truncated to FP32 (complex128: by integer bit
// operations, no FP64 instruction), relative error below 2^-20.  Its bits (sign 0) are
// monotone in the value: coarse bin = bits >> 20 (exponent + 3 mantissa bits), fine bin =
// (bits >> 9) & 2047 (fine bins are 2^-14 relative wide).  The K-th largest p32 lies in fine
// bin T = (b1 << 11) | b2; every element of the exact top K has p32 at or above fine bin
// T - 1 (the FP32 error is far below one fine bin), and every element below it has an exact
// key below the K-th one, so sorting the candidates by (exact key desc, index asc) gives the
// exact selection and tie order.
constexpr int kTkBins = 2048;
constexpr int kTkCap = 8192;  // candidates the one-block sort holds

struct TkState {
    int ok;                  // 1: fast path chosen (the exact pipeline then returns at once)
    unsigned int cnt;        // candidates collected (must follow ok)
    unsigned int b1, thr;    // coarse bin of the K-th value, threshold on bits >> 9
    unsigned long long above1, need1;
};

__device__ __forceinline__ float trunc_f32(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    if (e <= 0) return 0.0f;
    if (e >= 255) return __int_as_float(0x7F7FFFFF);
    return __uint_as_float((hi & 0x80000000u) | ((uint32_t)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}
__device__ __forceinline__ uint32_t p32_bits(double2 a) {
    const float x = trunc_f32(a.x), y = trunc_f32(a.y);
    return __float_as_uint(fmaf(x, x, y * y));
}
__device__ __forceinline__ uint32_t p32_bits(float2 a) { return __float_as_uint(fmaf(a.x, a.x, a.y * a.y)); }

template <typename V, int LEVEL>
__global__ void __launch_bounds__(256)
k_tk_hist(const V *__restrict__ psi, uint64_t n, const TkState *__restrict__ ts,
          unsigned long long *__restrict__ hist) {
    __shared__ unsigned int h[kTkBins];
    for (int i = threadIdx.x; i < kTkBins; i += 256) h[i] = 0;
    __syncthreads();
    const uint32_t b1 = LEVEL == 2 ? ts->b1 : 0u;
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (uint64_t)gridDim.x * 256) {
        const uint32_t b = p32_bits(psi[i]);
        if (LEVEL == 1) atomicAdd(&h[b >> 20], 1u);
        else if ((b >> 20) == b1) atomicAdd(&h[(b >> 9) & (kTkBins - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTkBins; i += 256)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

__global__ void k_tk_plan1(const unsigned long long *__restrict__ h1, unsigned long long K, TkState *ts) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long acc = 0;
    int b = kTkBins - 1;
    for (; b > 0; b--) {
        if (acc + h1[b] >= K) break;
        acc += h1[b];
    }
    ts->b1 = (unsigned int)b;
    ts->above1 = acc;
    ts->need1 = K - acc;
    ts->ok = 0;
    ts->cnt = 0;
}

__global__ void k_tk_plan2(const unsigned long long *__restrict__ h1, const unsigned long long *__restrict__ h2,
                           uint64_t n, TkState *ts) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long need = ts->need1;
    unsigned long long acc = 0;
    int b2 = kTkBins - 1;
    for (; b2 > 0; b2--) {
        if (acc + h2[b2] >= need) break;
        acc += h2[b2];
    }
    const uint32_t b1 = ts->b1, T = (b1 << 11) | (uint32_t)b2;
    unsigned long long c;
    if (b2 >= 1) {
        c = ts->above1;
        for (int f = b2 - 1; f < kTkBins; f++) c += h2[f];
    } else if (b1 >= 1) {
        c = ts->above1 + h1[b1] + h1[b1 - 1];  // bound: part of coarse bin b1 - 1 may join
    } else {
        c = n;
    }
    ts->thr = T >= 1 ? T - 1 : 0u;
    ts->ok = c <= (unsigned long long)kTkCap ? 1 : 0;
}

template <typename V>
__global__ void __launch_bounds__(256)
k_tk_collect(const V *__restrict__ psi, uint64_t n, TkState *__restrict__ ts,
             unsigned long long *__restrict__ ckey, unsigned long long *__restrict__ cidx) {
    if (!ts->ok) return;
    const uint32_t thr = ts->thr;
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (uint64_t)gridDim.x * 256) {
        const V a = psi[i];
        if ((p32_bits(a) >> 9) >= thr) {
            const unsigned int slot = atomicAdd(&ts->cnt, 1u);
            if (slot < (unsigned int)kTkCap) {
                ckey[slot] = key_of(a);
                cidx[slot] = i;
            }
        }
    }
}

// First-level block = 2^cb amplitudes: large enough that the block's combine step (cb + 1
// sums over 256 thread values) stays small beside the per-amplitude work, small enough to
// leave 2^12 blocks or more (several waves of resident blocks) from 24 qubits on.
int chunk_bits(int n) { return std::min(n, std::max(12, std::min(16, n - 12))); }

}  // namespace

void launch_set_zero_state(DeviceState &st) {
    const size_t B = st.dtype == QS_C128 ? 16 : 8;
    QS_CUDA(cudaMemsetAsync(st.psi, 0, B << st.n, st.stream));
    k_set_one<<<1, 1, 0, st.stream>>>(st.psi, st.dtype == QS_C128);
    QS_CUDA(cudaGetLastError());
    count_launch();
    st.known_zero = true;
}

void launch_scale(DeviceState &st, double f) {
    st.known_zero = false;
    const uint64_t n = 1ull << st.n;
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)device_sm_count() * 8);
    if (st.dtype == QS_C128) k_scale<double2, double><<<grid, 256, 0, st.stream>>>((double2 *)st.psi, n, f);
    else k_scale<float2, float><<<grid, 256, 0, st.stream>>>((float2 *)st.psi, n, (float)f);
    QS_CUDA(cudaGetLastError());
    count_launch();
}

namespace {

// Word-wise copy by a grid-stride loop (one of the two sides is mapped host memory); four
// loads in flight per thread, so a small grid still covers the link's latency.
template <typename W>
__global__ void __launch_bounds__(256) k_copy_words(const W *__restrict__ src, W *__restrict__ dst, uint64_t n) {
    constexpr int kUn = 4;
    const uint64_t stride = (uint64_t)gridDim.x * 256;
    uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
    for (; i + (kUn - 1) * stride < n; i += kUn * stride) {
        W v[kUn];
#pragma unroll
        for (int u = 0; u < kUn; u++) v[u] = src[i + u * stride];
#pragma unroll
        for (int u = 0; u < kUn; u++) dst[i + u * stride] = v[u];
    }
    for (; i < n; i += stride) dst[i] = src[i];
}

// Device address of [p, p + bytes) if the whole range is page-locked host memory mapped
// into this device's address space (first and last byte checked), else null.
const void *mapped_range(const void *p, size_t bytes) {
    cudaPointerAttributes a0{}, a1{};
    const char *last = (const char *)p + bytes - 1;
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess || cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
        return nullptr;
    if ((const char *)a1.devicePointer != (const char *)a0.devicePointer + (bytes - 1)) return nullptr;
    return a0.devicePointer;
}

}  // namespace

void copy_host(DeviceState &st, void *dst, const void *src, size_t bytes, bool to_device, int ctas) {
    if (to_device) st.known_zero = false;
    if (bytes == 0) return;
    constexpr size_t kMinKernelBytes = 4u << 20;
    const void *host = to_device ? src : dst;
    const void *mh = (ctas != kCopyEngines && bytes >= kMinKernelBytes) ? mapped_range(host, bytes) : nullptr;
    const char *s = to_device ? (const char *)mh : (const char *)src;
    char *d = to_device ? (char *)dst : (char *)mh;
    const uintptr_t align = (uintptr_t)s | (uintptr_t)d | (uintptr_t)bytes;
    if (mh && (align & 7u) == 0) {
        const int grid = ctas > 0 ? ctas : device_sm_count() * 8;
        if ((align & 15u) == 0)
            k_copy_words<int4><<<grid, 256, 0, st.stream>>>((const int4 *)s, (int4 *)d, bytes / 16);
        else
            k_copy_words<uint2><<<grid, 256, 0, st.stream>>>((const uint2 *)s, (uint2 *)d, bytes / 8);
        QS_CUDA(cudaGetLastError());
        count_launch();
        return;
    }
    QS_CUDA(cudaMemcpyAsync(dst, src, bytes, to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                            st.stream));
}

size_t scratch_expz_bytes(int n) { return expz_pipeline_doubles(n, chunk_bits(n)) * sizeof(double); }

// Norm and <Z_q> into out_dev (n + 1 doubles); the partials use st.scratch.
static void expz_launch(DeviceState &st, bool bits, double *out_dev) {
    ensure_scratch(st, scratch_expz_bytes(st.n));
    expz_pipeline(st.psi, st.dtype == QS_C128, st.n, chunk_bits(st.n), bits, (double *)st.scratch, out_dev,
                  st.stream);
}

void reduce_expz_async(DeviceState &st, double *out_dev) { expz_launch(st, true, out_dev); }

void reduce_norm_async(DeviceState &st, double *out_dev) { expz_launch(st, false, out_dev); }

void launch_scale_ratio(DeviceState &st, const double *norms_dev) {
    const uint64_t n = 1ull << st.n;
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)device_sm_count() * 8);
    if (st.dtype == QS_C128) k_scale_ratio<double2><<<grid, 256, 0, st.stream>>>((double2 *)st.psi, n, norms_dev);
    else k_scale_ratio<float2><<<grid, 256, 0, st.stream>>>((float2 *)st.psi, n, norms_dev);
    QS_CUDA(cudaGetLastError());
    count_launch();
}

void reduce_expz(DeviceState &st, double *norm, double *expz) {
    const int n = st.n;
    const bool bits = expz != nullptr;
    ensure_scratch(st, scratch_expz_bytes(n));
    double *out = (double *)st.scratch + expz_pipeline_doubles(n, chunk_bits(n)) - (n + 1);
    expz_launch(st, bits, out);
    std::vector<double> h(n + 1);
    QS_CUDA(cudaMemcpyAsync(h.data(), out, sizeof(double) * (bits ? n + 1 : 1), cudaMemcpyDeviceToHost, st.stream));
    QS_CUDA(cudaStreamSynchronize(st.stream));
    if (norm) *norm = h[0];
    if (bits)
        for (int q = 0; q < n; q++) expz[q] = h[1 + q];
}

namespace {
struct TopkLayout {
    size_t o_sel, o_hist, o_tie, o_gt, o_key, o_idx, o_oidx, o_oamp, o_ts, o_h1, o_h2, o_ckey, o_cidx, total;
};
TopkLayout topk_layout(int n, uint32_t K) {
    const int cb = std::min(n, 12);
    const uint64_t nblk = (1ull << n) >> cb;
    TopkLayout L{};
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    L.o_sel = carve(sizeof(SelState));
    L.o_hist = carve(sizeof(unsigned long long) * kBins);
    L.o_tie = carve(sizeof(unsigned int) * nblk);
    L.o_gt = carve(sizeof(unsigned int));
    L.o_key = carve(sizeof(unsigned long long) * K);
    L.o_idx = carve(sizeof(unsigned long long) * K);
    L.o_oidx = carve(sizeof(unsigned long long) * K);
    L.o_oamp = carve(sizeof(double) * 2 * K);
    L.o_ts = carve(sizeof(TkState));
    L.o_h1 = carve(sizeof(unsigned long long) * kTkBins);
    L.o_h2 = carve(sizeof(unsigned long long) * kTkBins);
    L.o_ckey = carve(sizeof(unsigned long long) * kTkCap);
    L.o_cidx = carve(sizeof(unsigned long long) * kTkCap);
    L.total = off;
    return L;
}
}  // namespace

size_t scratch_topk_bytes(int n, uint32_t k) { return topk_layout(n, k).total; }

// Launches the whole top-K pipeline; results to idx_dev / amp_dev (device).  The fast path
// (two histogram passes, one collection pass, one sort) is enqueued first; the exact radix
// pipeline follows and each of its kernels returns at once when the fast path was taken
// (a device flag), so nothing waits on the host.
void top_k_async(DeviceState &st, uint32_t K, uint64_t *idx_dev, double *amp_dev) {
    const int n = st.n;
    const uint64_t N = 1ull << n;
    if (K == 0) return;
    if (K > N || K > 4096) fail(QS_ERR_INVALID, "top-k: k exceeds min(2^n, 4096)");
    const int cb = std::min(n, 12);
    const uint64_t nblk = N >> cb;
    const TopkLayout TL = topk_layout(n, K);
    ensure_scratch(st, TL.total);
    char *base = (char *)st.scratch;
    const bool c128 = st.dtype == QS_C128;
    const int grid = (int)std::min<uint64_t>((N + 255) / 256, (uint64_t)device_sm_count() * 8);
    unsigned long long *oidx = (unsigned long long *)idx_dev;
    double *oamp = amp_dev;
    auto sort_launch = [&](const unsigned long long *key, const unsigned long long *idx, int P, int n_in,
                           const unsigned int *n_in_dev, const int *flag, int skip_when) {
        const size_t smem = sizeof(unsigned long long) * 2 * P;
        if (c128) {
            auto kern = k_topk_sort<double2>;
            QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<1, 1024, smem, st.stream>>>((const double2 *)st.psi, key, idx, (int)K, P, n_in, n_in_dev, oidx,
                                               oamp, flag, skip_when);
        } else {
            auto kern = k_topk_sort<float2>;
            QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<1, 1024, smem, st.stream>>>((const float2 *)st.psi, key, idx, (int)K, P, n_in, n_in_dev, oidx,
                                               oamp, flag, skip_when);
        }
        QS_CUDA(cudaGetLastError());
    };
    // ---- fast path
    TkState *ts = (TkState *)(base + TL.o_ts);
    unsigned long long *h1 = (unsigned long long *)(base + TL.o_h1), *h2 = (unsigned long long *)(base + TL.o_h2);
    unsigned long long *ckey = (unsigned long long *)(base + TL.o_ckey), *cidx = (unsigned long long *)(base + TL.o_cidx);
    QS_CUDA(cudaMemsetAsync(h1, 0, sizeof(unsigned long long) * kTkBins, st.stream));
    QS_CUDA(cudaMemsetAsync(h2, 0, sizeof(unsigned long long) * kTkBins, st.stream));
    if (c128) k_tk_hist<double2, 1><<<grid, 256, 0, st.stream>>>((const double2 *)st.psi, N, ts, h1);
    else k_tk_hist<float2, 1><<<grid, 256, 0, st.stream>>>((const float2 *)st.psi, N, ts, h1);
    k_tk_plan1<<<1, 1, 0, st.stream>>>(h1, (unsigned long long)K, ts);
    if (c128) k_tk_hist<double2, 2><<<grid, 256, 0, st.stream>>>((const double2 *)st.psi, N, ts, h2);
    else k_tk_hist<float2, 2><<<grid, 256, 0, st.stream>>>((const float2 *)st.psi, N, ts, h2);
    k_tk_plan2<<<1, 1, 0, st.stream>>>(h1, h2, N, ts);
    if (c128) k_tk_collect<double2><<<grid, 256, 0, st.stream>>>((const double2 *)st.psi, N, ts, ckey, cidx);
    else k_tk_collect<float2><<<grid, 256, 0, st.stream>>>((const float2 *)st.psi, N, ts, ckey, cidx);
    QS_CUDA(cudaGetLastError());
    sort_launch(ckey, cidx, kTkCap, -1, &ts->cnt, &ts->ok, 0);
    count_launch(6);
    // ---- exact radix pipeline (returns at once when ts->ok)
    const int *skip = &ts->ok;
    SelState *sel = (SelState *)(base + TL.o_sel);
    unsigned long long *hist = (unsigned long long *)(base + TL.o_hist);
    k_sel_init<<<1, 1, 0, st.stream>>>(sel, (unsigned long long)K, skip);
    count_launch();
    QS_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kBins, st.stream));
    QS_CUDA(cudaMemsetAsync(base + TL.o_gt, 0, sizeof(unsigned int), st.stream));
    // keys are non-negative doubles: bit 63 is always 0, digits cover bits 62..0
    int hi = 64;
    for (int shift = 63 - kDigitBits; hi > 0; shift -= kDigitBits) {
        const int sh = std::max(shift, 0);
        if (c128) k_sel_hist<double2><<<grid, 256, 0, st.stream>>>((const double2 *)st.psi, N, sel, hi, sh, hist, skip);
        else k_sel_hist<float2><<<grid, 256, 0, st.stream>>>((const float2 *)st.psi, N, sel, hi, sh, hist, skip);
        k_sel_pick<<<1, 1, 0, st.stream>>>(sel, hist, sh, skip);
        count_launch(2);
        hi = sh;
    }
    unsigned int *tie = (unsigned int *)(base + TL.o_tie);
    if (c128) k_tie_count<double2><<<(unsigned)nblk, 256, 0, st.stream>>>((const double2 *)st.psi, cb, sel, tie, skip);
    else k_tie_count<float2><<<(unsigned)nblk, 256, 0, st.stream>>>((const float2 *)st.psi, cb, sel, tie, skip);
    k_tie_scan<<<1, 1, 0, st.stream>>>(tie, nblk, skip);
    unsigned long long *gkey = (unsigned long long *)(base + TL.o_key), *gidx = (unsigned long long *)(base + TL.o_idx);
    if (c128)
        k_gather<double2><<<(unsigned)nblk, 256, 0, st.stream>>>((const double2 *)st.psi, cb, sel, K, tie,
                                                                   (unsigned int *)(base + TL.o_gt), gkey, gidx, skip);
    else
        k_gather<float2><<<(unsigned)nblk, 256, 0, st.stream>>>((const float2 *)st.psi, cb, sel, K, tie,
                                                                  (unsigned int *)(base + TL.o_gt), gkey, gidx, skip);
    QS_CUDA(cudaGetLastError());
    int P = 1;
    while (P < (int)K) P <<= 1;
    P = std::max(P, 2);
    sort_launch(gkey, gidx, P, (int)K, nullptr, skip, 1);
    count_launch(4);
}

void top_k(DeviceState &st, uint32_t K, uint64_t *idx, double *amp) {
    if (K == 0) return;
    if ((uint64_t)K > (1ull << st.n) || K > 4096) fail(QS_ERR_INVALID, "top-k: k exceeds min(2^n, 4096)");
    const TopkLayout TL = topk_layout(st.n, K);
    ensure_scratch(st, TL.total);
    char *base = (char *)st.scratch;
    uint64_t *oidx = (uint64_t *)(base + TL.o_oidx);
    double *oamp = (double *)(base + TL.o_oamp);
    top_k_async(st, K, oidx, oamp);
    QS_CUDA(cudaMemcpyAsync(idx, oidx, sizeof(uint64_t) * K, cudaMemcpyDeviceToHost, st.stream));
    QS_CUDA(cudaMemcpyAsync(amp, oamp, sizeof(double) * 2 * K, cudaMemcpyDeviceToHost, st.stream));
    QS_CUDA(cudaStreamSynchronize(st.stream));
}

// ---------------------------------------------------------------------------------
// Allocation-free variant of the norm / <Z_q> reduction.
//
// Some callers cannot call cudaMalloc: for example a host program that has handed all of
// the device's memory to its own pool allocator, or a latency-critical loop that cannot
// afford the implicit device synchronisation and unbounded latency of cudaMalloc.  This
// entry point allocates nothing.  Its scratch is the file-scope device array below, of a
// fixed size (kNoAllocScratchDoubles doubles, about 2.5 MB), which every GPU that loads
// the library holds until the process exits.  The reduction kernels are the same as
// above; only the block size is chosen so that at most 2^14 blocks write partial sums.

namespace {

constexpr int kNoAllocMaxQubits = 32;
constexpr int kNoAllocMaxBlockBits = 14;
// partials: 2^14 blocks x (cb + 1 <= 19) doubles, then the n + 1 outputs
constexpr size_t kNoAllocScratchDoubles = ((size_t)1 << kNoAllocMaxBlockBits) * 19 + 2048 + 64;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[64] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up once per device and
// kept; a cudaDeviceReset of that device would leave the kept address stale).
double *noalloc_scratch() {
    int dev = 0;
    QS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(QS_ERR_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        QS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = (double *)p;
    }
    return g_noalloc_ptr[dev];
}

}  // namespace

}  // namespace qs

extern "C" int qs_expectation_z_noalloc(const void *dev_psi, int n_qubits, qs_dtype dt, void *stream,
                                        double *out_expz, double *out_norm) {
    using namespace qs;
    QS_API_BEGIN
    if (!dev_psi || (!out_expz && !out_norm)) fail(QS_ERR_INVALID, "NULL argument");
    if (dt != QS_C64 && dt != QS_C128) fail(QS_ERR_INVALID, "unknown dtype");
    if (n_qubits < 1 || n_qubits > kNoAllocMaxQubits)
        fail(QS_ERR_INVALID, "qs_expectation_z_noalloc takes 1 to 32 qubits (fixed static scratch of " +
                                 std::to_string(kNoAllocScratchDoubles) + " doubles)");
    const int n = n_qubits;
    const int cb = std::min(n, std::max(chunk_bits(n), n - kNoAllocMaxBlockBits));
    const size_t need = expz_pipeline_doubles(n, cb);
    if (need > kNoAllocScratchDoubles) fail(QS_ERR_INVALID, "static scratch too small");
    double *scratch = noalloc_scratch();
    double *out = scratch + need - (n + 1);
    cudaStream_t st = (cudaStream_t)stream;
    // every partial a level reads is written by the level before: nothing to clear
    expz_pipeline(dev_psi, dt == QS_C128, n, cb, true, scratch, out, st);
    double h[kNoAllocMaxQubits + 1];
    QS_CUDA(cudaMemcpyAsync(h, out, sizeof(double) * (n + 1), cudaMemcpyDeviceToHost, st));
    QS_CUDA(cudaStreamSynchronize(st));
    if (out_norm) *out_norm = h[0];
    if (out_expz)
        for (int q = 0; q < n; q++) out_expz[q] = h[1 + q];
    QS_API_END
}

