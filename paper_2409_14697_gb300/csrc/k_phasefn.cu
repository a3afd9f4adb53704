// Merged diagonal run (QueenV2 Sec. III-A tier 2, "infinite" diagonal gate fusion): one
// pass over the state multiplies every amplitude by its phase-table entry (phasefn.h).
//
// A warp owns units of 2^9 consecutive amplitudes: lane l and register r hold amplitude
// (unit << 9) | (r << 5) | l, so every load and store of a warp is 32 consecutive
// amplitudes, and bits 5..8 of the index vary over a thread's 16 registers while every
// other bit is the same for all of them.  Group counts: a weight group is a popcount of the
// thread-uniform bits plus a popcount of the register bits; a pair group counts pairs whose
// two bits are both set, scalar for pairs on uniform bits and in 12 bit planes (a ripple
// counter over the 16 registers at once) for pairs that touch register bits.
#include <algorithm>

#include "ixmath.cuh"
#include "kops.cuh"
#include "phasefn.h"

namespace qs {
namespace {

constexpr int kPfThreads = 256;
constexpr int kPfRegBits = 4;
constexpr int kPfRegs = 1 << kPfRegBits;
constexpr int kPfUnitBits = 5 + kPfRegBits;
constexpr int kPfPlanes = 12;       // counts up to 4095 (kPfMaxTable)
constexpr int kPfMaxPairs = 8192;   // pair list staged in shared memory (32 KiB)

struct PfGroupDev {
    int32_t kind;
    int32_t stride;
    int32_t pair_off;
    int32_t npairs;
    uint64_t mask;
};
struct PfArgs {
    int32_t ngroups;
    int32_t table_size;
    int32_t total_pairs;
    int32_t pad;
    uint64_t n_units;
    PfGroupDev g[kPfMaxGroups];
};

// bit r of the result = bit q of the amplitude in register r (16 registers)
__device__ __forceinline__ uint32_t pf_mask(int q, uint64_t xu) {
    switch (q) {
    case 5: return 0xAAAAu;
    case 6: return 0xCCCCu;
    case 7: return 0xF0F0u;
    case 8: return 0xFF00u;
    default: return ((xu >> q) & 1ull) ? 0xFFFFu : 0u;
    }
}

template <typename T>
__device__ __forceinline__ typename C2T<T>::type pf_cmul(typename C2T<T>::type a, typename C2T<T>::type f) {
    typename C2T<T>::type y;
    const T pr = -a.y * f.y, pi = a.x * f.y;
    y.x = fma(a.x, f.x, pr);
    y.y = fma(a.y, f.x, pi);
    return y;
}

// complex128 with integer products (QS_PREC_IX64): the factor is decoded per amplitude;
// registers 0, 4, 8 and 12 take the native FP64 product, so both pipes work.
__device__ __forceinline__ double2 pf_cmul_ix(double2 a, double2 f) {
    const ix::Num x[2] = {ix::decode(a.x), ix::decode(a.y)};
    double y[2];
    ix::cmul<0>(f.x, f.y, x, y);
    return make_double2(y[0], y[1]);
}

template <typename T, bool IX>
__global__ void __launch_bounds__(kPfThreads)
k_phasefn(typename C2T<T>::type *__restrict__ psi, const PfArgs a, const uint32_t *__restrict__ pairs,
          const typename C2T<T>::type *__restrict__ table) {
    using V = typename C2T<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    V *s_tab = (V *)smem;
    uint32_t *s_pairs = (uint32_t *)(s_tab + a.table_size);
    for (int i = threadIdx.x; i < a.table_size; i += blockDim.x) s_tab[i] = table[i];
    for (int i = threadIdx.x; i < a.total_pairs; i += blockDim.x) s_pairs[i] = pairs[i];
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t wstep = (uint64_t)gridDim.x * (kPfThreads / 32);
    for (uint64_t u = (uint64_t)blockIdx.x * (kPfThreads / 32) + warp; u < a.n_units; u += wstep) {
        const uint64_t xu = (u << kPfUnitBits) | lane;  // the register bits 5..8 are zero
        V v[kPfRegs];
#pragma unroll
        for (int r = 0; r < kPfRegs; r++) v[r] = psi[xu + ((uint64_t)r << 5)];
        int idx[kPfRegs];
#pragma unroll
        for (int r = 0; r < kPfRegs; r++) idx[r] = 0;
        for (int gi = 0; gi < a.ngroups; gi++) {
            const PfGroupDev &G = a.g[gi];
            if (G.kind == PF_WEIGHT) {
                const int cu = __popcll(xu & G.mask);
                const uint32_t mr = (uint32_t)(G.mask >> 5) & (uint32_t)(kPfRegs - 1);
#pragma unroll
                for (int r = 0; r < kPfRegs; r++) idx[r] += (cu + __popc((uint32_t)r & mr)) * G.stride;
            } else {
                int cu = 0;
                uint32_t c[kPfPlanes];
#pragma unroll
                for (int k = 0; k < kPfPlanes; k++) c[k] = 0;
                for (int p = 0; p < G.npairs; p++) {
                    const uint32_t e = s_pairs[G.pair_off + p];
                    const uint32_t M = pf_mask((int)(e & 63u), xu) & pf_mask((int)(e >> 8), xu);
                    if (M == 0xFFFFu) {
                        cu++;
                    } else if (M) {
                        uint32_t cy = M;
#pragma unroll
                        for (int k = 0; k < kPfPlanes; k++) {
                            const uint32_t t = c[k] & cy;
                            c[k] ^= cy;
                            cy = t;
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < kPfRegs; r++) {
                    int cnt = cu;
#pragma unroll
                    for (int k = 0; k < kPfPlanes; k++) cnt += (int)((c[k] >> r) & 1u) << k;
                    idx[r] += cnt * G.stride;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kPfRegs; r++) {
            if constexpr (IX) {
                psi[xu + ((uint64_t)r << 5)] =
                    (r % 4 == 0) ? pf_cmul<T>(v[r], s_tab[idx[r]]) : pf_cmul_ix(v[r], s_tab[idx[r]]);
            } else {
                psi[xu + ((uint64_t)r << 5)] = pf_cmul<T>(v[r], s_tab[idx[r]]);
            }
        }
    }
}

template <typename T, bool IX>
void launch_t(DeviceState &st, const PhaseFn &pf) {
    using V = typename C2T<T>::type;
    PfArgs a{};
    a.ngroups = (int32_t)pf.groups.size();
    a.table_size = (int32_t)pf.table.size();
    a.n_units = 1ull << (st.n - kPfUnitBits);
    std::vector<uint32_t> pl;
    for (size_t i = 0; i < pf.groups.size(); i++) {
        const PfGroup &g = pf.groups[i];
        PfGroupDev &d = a.g[i];
        d.kind = g.kind;
        d.stride = g.stride;
        d.mask = g.mask;
        d.pair_off = (int32_t)pl.size();
        d.npairs = (int32_t)g.pairs.size();
        for (const auto &p : g.pairs) pl.push_back((uint32_t)p.first | (uint32_t)p.second << 8);
    }
    if ((int)pl.size() > kPfMaxPairs) fail(QS_ERR_UNSUPPORTED, "phase function with too many qubit pairs");
    a.total_pairs = (int32_t)pl.size();
    if (pl.empty()) pl.push_back(0);
    std::vector<V> tab(pf.table.size());
    for (size_t i = 0; i < tab.size(); i++) {
        tab[i].x = (T)pf.table[i].real();
        tab[i].y = (T)pf.table[i].imag();
    }
    const V *d_tab = (const V *)upload_params(st, tab.data(), tab.size() * sizeof(V));
    const uint32_t *d_pairs = (const uint32_t *)upload_params(st, pl.data(), pl.size() * sizeof(uint32_t));
    const size_t smem = tab.size() * sizeof(V) + (size_t)a.total_pairs * sizeof(uint32_t);
    auto kern = k_phasefn<T, IX>;
    static bool attr = false;
    if (!attr) {
        QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
        attr = true;
    }
    const uint64_t blocks = (a.n_units + kPfThreads / 32 - 1) / (kPfThreads / 32);
    const int grid = persistent_grid((const void *)kern, kPfThreads, smem, blocks);
    kern<<<grid, kPfThreads, smem, st.stream>>>((V *)st.psi, a, d_pairs, d_tab);
    QS_CUDA(cudaGetLastError());
    count_launch();
}

}  // namespace

bool phasefn_supported(int n) { return n >= kPfUnitBits; }

void launch_phasefn(DeviceState &st, const Op &op) {
    if (op.kind != K_PHASEFN || !op.pf) fail(QS_ERR_INVALID, "not a phase function");
    if (!phasefn_supported(st.n)) fail(QS_ERR_UNSUPPORTED, "phase functions need at least 9 qubits");
    if (st.dtype == QS_C128 && st.ix) launch_t<double, true>(st, *op.pf);
    else if (st.dtype == QS_C128) launch_t<double, false>(st, *op.pf);
    else launch_t<float, false>(st, *op.pf);
}

}  // namespace qs
