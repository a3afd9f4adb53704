// Tensor Product Booster, last step (QueenV2 Sec. III-A tier 1): the state of a circuit
// prefix whose gates split into independent qubit groups is the tensor product of the
// groups' sub-states, a[x] = prod_g T_g[pext(x, M_g)], written in one pass over the
// state (write only).  The sub-states T_g (at most 2^17 amplitudes each, resident in L2)
// were built by the ordinary executor on small states; tpb.cpp finds the prefix.
//
// Work split: a warp owns runs of 32 x kTpbRegs consecutive amplitudes; lane l and
// register r hold amplitude base + 32 r + l, so every store of a warp is 32 consecutive
// amplitudes.  pext is additive over disjoint bit sets, so the table index of a group is
// pext(base + 32 r, M_g) (warp-uniform, from per-byte lookup tables in shared memory)
// plus pext(l, M_g) (per lane, computed once).
#include <algorithm>

#include "kops.cuh"
#include "qs_internal.h"

namespace qs {
namespace {

constexpr int kTpbThreads = 256;
constexpr int kTpbRegs = 8;
constexpr int kTpbRunBits = 5 + 3;      // 32 lanes x 8 registers
constexpr int kTpbBytes = 5;            // index bytes covered by the lookup tables (40 bits)

struct TpbArgs {
    const void *table[kTpbMaxGroups];
    uint64_t mask[kTpbMaxGroups];
    int32_t groups;
    int32_t n;
};

__device__ __forceinline__ uint32_t pext_bits(uint64_t x, uint64_t m) {
    uint32_t r = 0;
    int o = 0;
    while (m) {
        const int b = __ffsll((long long)m) - 1;
        r |= (uint32_t)((x >> b) & 1ull) << o;
        o++;
        m &= m - 1;
    }
    return r;
}

template <typename T>
__device__ __forceinline__ typename C2T<T>::type tpb_cmul(typename C2T<T>::type a, typename C2T<T>::type b) {
    typename C2T<T>::type y;
    y.x = fma(a.x, b.x, -a.y * b.y);
    y.y = fma(a.x, b.y, a.y * b.x);
    return y;
}

template <typename T, int G>
__global__ void __launch_bounds__(kTpbThreads) k_tpb(typename C2T<T>::type *__restrict__ psi, TpbArgs a) {
    using V = typename C2T<T>::type;
    __shared__ uint32_t lut[G][kTpbBytes][256];
    for (int e = threadIdx.x; e < G * kTpbBytes * 256; e += kTpbThreads) {
        const int g = e / (kTpbBytes * 256), b = (e / 256) % kTpbBytes, v = e % 256;
        lut[g][b][v] = pext_bits((uint64_t)v << (8 * b), a.mask[g]);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint32_t lo[G];
    const V *tab[G];
#pragma unroll
    for (int g = 0; g < G; g++) {
        lo[g] = pext_bits((uint64_t)lane, a.mask[g]);
        tab[g] = (const V *)a.table[g];
    }
    const uint64_t n_runs = (1ull << a.n) >> kTpbRunBits;
    const uint64_t warps = (uint64_t)gridDim.x * (kTpbThreads / 32);
    for (uint64_t run = (uint64_t)blockIdx.x * (kTpbThreads / 32) + threadIdx.x / 32; run < n_runs; run += warps) {
        const uint64_t base = run << kTpbRunBits;
        V out[kTpbRegs];
#pragma unroll
        for (int r = 0; r < kTpbRegs; r++) {
            const uint64_t hi = base + 32ull * r;
            V acc;
#pragma unroll
            for (int g = 0; g < G; g++) {
                uint32_t idx = lo[g];
#pragma unroll
                for (int b = 0; b < kTpbBytes; b++) idx += lut[g][b][(hi >> (8 * b)) & 0xFF];
                const V t = tab[g][idx];
                acc = g == 0 ? t : tpb_cmul<T>(acc, t);
            }
            out[r] = acc;
        }
#pragma unroll
        for (int r = 0; r < kTpbRegs; r++) psi[base + 32ull * r + lane] = out[r];
    }
}

template <typename T, int G>
void launch_g(DeviceState &st, const TpbArgs &a, uint64_t blocks) {
    const int grid = persistent_grid((const void *)k_tpb<T, G>, kTpbThreads, 0, blocks);
    k_tpb<T, G><<<grid, kTpbThreads, 0, st.stream>>>((typename C2T<T>::type *)st.psi, a);
}

template <typename T>
void launch_groups(DeviceState &st, const TpbArgs &a, uint64_t blocks) {
    static_assert(kTpbMaxGroups == 4, "one instance per group count");
    switch (a.groups) {
    case 1: launch_g<T, 1>(st, a, blocks); break;
    case 2: launch_g<T, 2>(st, a, blocks); break;
    case 3: launch_g<T, 3>(st, a, blocks); break;
    default: launch_g<T, 4>(st, a, blocks); break;
    }
}

}  // namespace

void launch_tpb_product(DeviceState &st, const void *const *tables, const uint64_t *masks, int groups) {
    if (groups < 1 || groups > kTpbMaxGroups) fail(QS_ERR_INVALID, "internal: tensor-product group count");
    if (st.n < kTpbRunBits || st.n > 8 * kTpbBytes) fail(QS_ERR_INVALID, "internal: tensor-product state size");
    TpbArgs a{};
    uint64_t all = 0;
    for (int g = 0; g < groups; g++) {
        a.table[g] = tables[g];
        a.mask[g] = masks[g];
        if (masks[g] & all) fail(QS_ERR_INVALID, "internal: overlapping tensor-product groups");
        all |= masks[g];
    }
    if (all != ((1ull << st.n) - 1ull)) fail(QS_ERR_INVALID, "internal: tensor-product groups do not cover the state");
    a.groups = groups;
    a.n = st.n;
    const uint64_t warps_needed = (1ull << st.n) >> kTpbRunBits;
    const uint64_t blocks = (warps_needed + kTpbThreads / 32 - 1) / (kTpbThreads / 32);
    if (st.dtype == QS_C128) launch_groups<double>(st, a, blocks);
    else launch_groups<float>(st, a, blocks);
    QS_CUDA(cudaGetLastError());
    count_launch();
}

}  // namespace qs
