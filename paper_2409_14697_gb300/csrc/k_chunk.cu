// K2: in-shared-memory chunk pass ("in-cache operations", QueenV2 Sec. II-B; the
// block-by-block all-in-cache module, Sec. III-B).
//
// A pass owns a set L of m "local" qubits: bits 0..c0-1 (contiguous runs of 2^c0
// amplitudes in HBM) plus m - c0 higher bits chosen by the planner.  Every CTA takes
// tiles t in [0, 2^(n-m)): the tile is the 2^m amplitudes whose non-local bits spell t
// (the non-local bits are deposited from t, the local ones from the in-tile index, the
// PDEP/PEXT-style addressing of Sec. III-B).  The tile is staged into shared memory by
// TMA bulk copies (cp.async.bulk, one per contiguous run, completion on an mbarrier),
// every op of the pass is applied on tile-local bit positions (Eq. 2 / Eq. 3 groups),
// and the tile is written back once by TMA bulk stores.  One full HBM read + write per
// pass, however many ops it holds.
#include <algorithm>
#include <type_traits>

#include "chunk.h"
#include "kops.cuh"
#include "ptx.cuh"
#include "tile_ops.cuh"

namespace qs {
namespace {

constexpr int kChunkThreads = kTileThreads;
// Dynamic shared memory of a staged pass (tile + program): two CTAs per SM must fit.
constexpr size_t kStagedSmemLimit = 104 * 1024;

// Global amplitude index of tile t with its local bits zero.
__device__ __forceinline__ uint64_t tile_base(uint64_t t, const ChunkArgs &a) {
    uint64_t base = t << a.c0;
    for (int j = 0; j < a.nlh; j++) {
        const int b = a.lhigh[j];
        base = ((base >> b) << (b + 1)) | (base & ((1ull << b) - 1ull));
    }
    return base;
}

// Reals of the table as FP64 (plain, or (hi, lo) float pairs with double-float passes).
template <bool DF> struct TabReal;
template <> struct TabReal<false> {
    template <typename T> static __device__ __forceinline__ double get(const T *p, int i) { return (double)p[i]; }
    template <typename T> static __device__ __forceinline__ void put(T *p, int i, double v) { p[i] = (T)v; }
};
template <> struct TabReal<true> {
    template <typename T> static __device__ __forceinline__ double get(const T *p, int i) {
        const df::F2 x = ((const df::F2 *)p)[i];
        return df::join(x.h, x.l);
    }
    template <typename T> static __device__ __forceinline__ void put(T *p, int i, double v) {
        ((df::F2 *)p)[i] = df::split(v);
    }
};

// Per-tile table of an F_CDIAGK / F_HCDIAGK block with non-local terms (op.nt > 0): the table with,
// for every term whose global qubit is 1 in this tile, its factor on the entries it covers.
// Warp w + 1 multiplies up the terms of table bit w (warp 0: the terms on every entry), in
// a fixed butterfly; then each entry takes the factors of its set bits.  Factors without
// terms (op.off[0]) are skipped: a QFT target's terms all sit on its control, so one warp
// works.  FP64 throughout.
// src: the op's reals; dst: scratch for the 2 * 2^k table reals (may equal src).
template <bool DF, typename T>
__device__ void fold_hi_terms(const KOp &op, const T *src, T *dst, uint64_t base) {
    __shared__ double s_f[2 * 8];  // [0]: every entry, [1 + b]: entries with table bit b
    using R = TabReal<DF>;
    const int kt = op.k, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ne = 1u << kt;
    const uint64_t with_terms = op.off[0];  // bit w: factor w has terms
    if (warp <= kt && warp < 8 && !((with_terms >> warp) & 1ull)) {
        if (lane == 0) {
            s_f[2 * warp] = 1.0;
            s_f[2 * warp + 1] = 0.0;
        }
    } else if (warp <= kt && warp < 8) {
        const int tb = warp - 1;
        double fr = 1.0, fi = 0.0;
        for (int i = lane; i < op.nt; i += 32) {
            const int o = (int)(2 * ne) + 4 * i;
            if ((int)R::get(src, o) != tb || !((base >> (int)R::get(src, o + 1)) & 1ull)) continue;
            const double gr = R::get(src, o + 2), gi = R::get(src, o + 3);
            const double r = fr * gr - fi * gi;
            fi = fr * gi + fi * gr;
            fr = r;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const double gr = __shfl_xor_sync(0xffffffffu, fr, d), gi = __shfl_xor_sync(0xffffffffu, fi, d);
            const double r = fr * gr - fi * gi;
            fi = fr * gi + fi * gr;
            fr = r;
        }
        if (lane == 0) {
            s_f[2 * warp] = fr;
            s_f[2 * warp + 1] = fi;
        }
    }
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < ne; s += blockDim.x) {
        double vr = R::get(src, 2 * s), vi = R::get(src, 2 * s + 1);
        for (int w = 0; w <= kt; w++) {
            if (!((with_terms >> w) & 1ull) || (w > 0 && !((s >> (w - 1)) & 1u))) continue;
            const double gr = s_f[2 * w], gi = s_f[2 * w + 1];
            const double r = vr * gr - vi * gi;
            vi = vr * gi + vi * gr;
            vr = r;
        }
        R::put(dst, 2 * s, vr);
        R::put(dst, 2 * s + 1, vi);
    }
    __syncthreads();
}

// DF: complex128 with double-float arithmetic; mats then holds (hi, lo) float pairs.
// IX: complex128 one-qubit dense ops and constant diagonal ops in integer products
// (QS_PREC_IX64).
template <typename T, bool DF, bool IX>
__global__ void __launch_bounds__(kChunkThreads, 2)
k_chunk(typename C2T<T>::type *__restrict__ psi, const ChunkArgs a, const KOp *__restrict__ ops,
        const T *__restrict__ mats, int *__restrict__ err) {
    using V = typename C2T<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V *tile = (V *)smem_raw;
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    __shared__ KOp s_op;
    __shared__ T s_m[kMaxOpReals];
    __shared__ double s_fb[DF ? kMaxOpReals : 1];
    const uint32_t nruns = 1u << (a.m - a.c0);
    const uint32_t run_bytes = (uint32_t)sizeof(V) << a.c0;
    const uint32_t tile_bytes = (uint32_t)sizeof(V) << a.m;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
    }
    // staged: the whole pass program is copied once per CTA (tiles then need one barrier
    // per op instead of three, and no global reads of ops)
    const KOp *st_ops = (const KOp *)(smem_raw + a.ops_off);
    const T *st_m = (const T *)(smem_raw + a.reals_off);
    if (a.staged) {
        const uint32_t *src = (const uint32_t *)ops;
        uint32_t *dst = (uint32_t *)(smem_raw + a.ops_off);
        const uint32_t nw = (uint32_t)a.n_ops * (uint32_t)(sizeof(KOp) / 4);
        for (uint32_t j = threadIdx.x; j < nw; j += blockDim.x) dst[j] = src[j];
        T *dm = (T *)(smem_raw + a.reals_off);
        for (uint32_t j = threadIdx.x; j < a.n_reals; j += blockDim.x) dm[j] = mats[j];
    }
    __syncthreads();
    uint32_t phase = 0;
    for (uint64_t t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        uint64_t base = tile_base(t, a);
        if (threadIdx.x == 0) ptx::mbar_arrive_expect_tx(&bar, tile_bytes);
        __syncthreads();
        for (uint32_t r = threadIdx.x; r < nruns; r += blockDim.x) {
            uint64_t off = 0;
            for (int j = 0; j < a.nlh; j++) off |= (uint64_t)((r >> j) & 1u) << a.lhigh[j];
            ptx::bulk_g2s(tile + ((uint64_t)r << a.c0), psi + (base | off), run_bytes, &bar);
        }
        if (!ptx::mbar_wait_bounded(&bar, phase, ptx::kWaitLimitNs)) {
            abort_flag = 1;
            // copies may still be in flight: one more bounded wait before leaving
            ptx::mbar_wait_bounded(&bar, phase, ptx::kWaitLimitNs);
        }
        phase ^= 1u;
        __syncthreads();
        if (abort_flag) {
            if (threadIdx.x == 0) atomicExch(err, QS_ERR_TIMEOUT);
            break;
        }
        if constexpr (DF) {  // amplitudes as float pairs for the whole pass
            df_tile_split((double2 *)tile, a.m);
            __syncthreads();
        }
        // one call site of the op code (it is large: register phases)
        for (int i = 0; i < a.n_ops; i++) {
            const KOp *op;
            const T *om;
            if (a.staged) {
                op = st_ops + i;
                om = st_m + op->mat;
            } else {
                if (threadIdx.x == 0) s_op = ops[i];
                __syncthreads();
                for (int j = threadIdx.x; j < s_op.nmat; j += blockDim.x) s_m[j] = mats[s_op.mat + j];
                __syncthreads();
                op = &s_op;
                om = s_m;
            }
            if constexpr (std::is_same<T, double>::value) {  // complex128 passes only
                if ((op->fkind == F_CDIAGK || op->fkind == F_HCDIAGK) && op->nt > 0) {
                    fold_hi_terms<DF>(*op, om, s_m, tile_base(t, a));
                    om = s_m;
                }
            }
            if constexpr (DF) apply_op_dftile((double2 *)tile, *op, (const df::F2 *)om, s_fb, a.m);
            else apply_op_smem<T, true, IX>(tile, *op, om, a.m);
            __syncthreads();
        }
        if constexpr (DF) {
            df_tile_join((double2 *)tile, a.m);
            __syncthreads();
        }
        ptx::fence_proxy_async_smem();
        __syncthreads();
        // the write-back addresses are rebuilt rather than kept live through the ops
        // (register pressure of the complex64 register phases)
        asm volatile("" ::: "memory");
        base = tile_base(t, a);
        for (uint32_t r = threadIdx.x; r < nruns; r += blockDim.x) {
            uint64_t off = 0;
            for (int j = 0; j < a.nlh; j++) off |= (uint64_t)((r >> j) & 1u) << a.lhigh[j];
            ptx::bulk_s2g(psi + (base | off), tile + ((uint64_t)r << a.c0), run_bytes);
        }
        ptx::bulk_commit();
        ptx::bulk_wait_read_all();
        __syncthreads();
    }
    ptx::bulk_wait_all();
}

template <typename T, bool DF, bool IX>
void launch_t(DeviceState &st, const ChunkArgs &a, const std::vector<KOp> &kops, const std::vector<double> &mats) {
    const KOp *d_ops = (const KOp *)upload_params(st, kops.data(), kops.size() * sizeof(KOp));
    const T *d_m;
    if constexpr (DF) {
        // every real as a (hi, lo) float pair, same indices as the FP64 table
        std::vector<float> pm(2 * std::max<size_t>(mats.size(), 1));
        for (size_t i = 0; i < mats.size(); i++) {
            pm[2 * i] = (float)mats[i];
            pm[2 * i + 1] = (float)(mats[i] - (double)pm[2 * i]);
        }
        d_m = (const T *)upload_params(st, pm.data(), pm.size() * sizeof(float));
    } else {
        std::vector<T> tm(std::max<size_t>(mats.size(), 2));
        for (size_t i = 0; i < mats.size(); i++) tm[i] = (T)mats[i];
        d_m = (const T *)upload_params(st, tm.data(), tm.size() * sizeof(T));
    }
    using V = typename C2T<T>::type;
    // stage the pass program after the tile when two CTAs per SM still fit
    ChunkArgs ca = a;
    const size_t tile_bytes = sizeof(V) << a.m;
    const size_t ops_bytes = kops.size() * sizeof(KOp);
    const size_t reals_bytes = (DF ? 2 * sizeof(float) : sizeof(T)) * mats.size();
    size_t smem = tile_bytes;
    ca.ops_off = (uint32_t)tile_bytes;
    ca.reals_off = (uint32_t)(tile_bytes + ops_bytes);
    ca.n_reals = (uint32_t)mats.size();
    ca.staged = tile_bytes + ops_bytes + reals_bytes <= kStagedSmemLimit ? 1 : 0;
    if (ca.staged) smem = (tile_bytes + ops_bytes + reals_bytes + 15) / 16 * 16;
    auto kern = k_chunk<T, DF, IX>;
    static bool attr_set = false;
    if (!attr_set) {
        QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        // the whole unified L1 as shared memory: two CTAs of up to ~104 KB per SM
        QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
        attr_set = true;
    }
    const int grid = persistent_grid((const void *)kern, kChunkThreads, smem, a.n_tiles);
    kern<<<grid, kChunkThreads, smem, st.stream>>>((V *)st.psi, ca, d_ops, d_m, st.dev_err);
    QS_CUDA(cudaGetLastError());
    count_launch();
}

}  // namespace

void launch_chunk_pass(DeviceState &st, uint64_t lmask, const std::vector<KOp> &kops,
                       const std::vector<double> &mats) {
    ChunkArgs a{};
    const int n = st.n;
    a.m = __builtin_popcountll(lmask);
    a.c0 = 0;
    while (a.c0 < n && ((lmask >> a.c0) & 1ull)) a.c0++;
    a.nlh = 0;
    for (int b = a.c0; b < n; b++)
        if ((lmask >> b) & 1ull) a.lhigh[a.nlh++] = b;
    a.n_tiles = 1ull << (n - a.m);
    a.n_ops = (int)kops.size();
    const size_t B = st.dtype == QS_C128 ? 16 : 8;
    if ((B << a.c0) % 16 != 0) fail(QS_ERR_INVALID, "chunk runs must be multiples of 16 bytes");
    if ((B << a.m) > 200 * 1024) fail(QS_ERR_INVALID, "chunk tile exceeds shared memory");
    if (st.dtype == QS_C128) {
        if (st.prec == QS_PREC_DF32) launch_t<double, true, false>(st, a, kops, mats);
        else if (st.ix) launch_t<double, false, true>(st, a, kops, mats);
        else launch_t<double, false, false>(st, a, kops, mats);
    } else {
        launch_t<float, false, false>(st, a, kops, mats);
    }
}

}  // namespace qs
