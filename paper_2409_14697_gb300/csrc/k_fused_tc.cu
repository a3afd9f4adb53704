// K3: fused dense blocks on the tensor cores (tcgen05), inside in-cache chunk passes.
//
// Gate fusion (QueenV2 Sec. II-B, Sec. III-A tier 5) merges runs of gates into one dense
// 2^k x 2^k block; applying it to every group of 2^k amplitudes (Eq. 2/3 generalised) is a
// complex matrix product over all groups.  Written over the reals with interleaved
// (re, im) columns it is the real GEMM
//     Y[g][2r + c] = sum_{s, c'} X[g][2s + c'] R[2r + c][2s + c'],
//     R = [[Re G, -Im G], [Im G, Re G]] per complex entry,
// with M = groups, N = K = 2^(k+1).  A complex64 chunk tile of 2^m amplitudes (m = 13)
// holds 2^(m-k) groups, i.e. 2^(m-k-7) MMA row tiles of 128 groups.
//
// Per tile: every thread owns one group (one TMEM lane) and writes its 2^(k+1) reals into
// TMEM with tcgen05.st, split into TF32 high and low parts (x = hi + lo, hi = x with the
// low 13 mantissa bits cleared); one thread issues tcgen05.mma kind::tf32 with A in TMEM
// and B = R (hi and lo parts, K-major canonical layout) in shared memory:
// D = A_hi B_hi + A_hi B_lo + A_lo B_hi (3xTF32 split products, FP32 accumulation in TMEM);
// the MMAs are committed to an mbarrier; each thread reads its row of D back with
// tcgen05.ld and writes the group's new amplitudes into the tile.  TMEM: 512 columns
// (A_hi, A_lo and D, 3 x 2^(m+1) / 128 <= 384 columns, rounded up), one CTA per SM.
#include <algorithm>
#include <cstring>

#include "chunk.h"
#include "kops.cuh"
#include "ptx.cuh"
#include "tc.cuh"
#include "tile_ops.cuh"

namespace qs {
namespace {

constexpr int kTcThreads = 256;
constexpr uint32_t kTmemCols = 512;

// Round a float to the nearest TF32 value (10 explicit mantissa bits; ties to even).
// The tensor cores read only the top 19 bits of a TF32 operand, i.e. they truncate; an
// operand that is already a TF32 value is read exactly, so rounding here keeps the split
// x = hi + lo unbiased (truncation would bias every product toward zero and the state's
// norm would drift over many blocks).
__device__ __forceinline__ uint32_t tf32_rn(float x) {
    const uint32_t b = __float_as_uint(x);
    return (b + 0x0FFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
}

// Rotates 8 complex values: out[j] = in[(j + sh) & 7] for sh in 0..7 (3 select stages).
__device__ __forceinline__ void rot8(float2 (&v)[8], int sh) {
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const int k = 1 << b;
        if ((sh >> b) & 1) {
            float2 t[8];
#pragma unroll
            for (int j = 0; j < 8; j++) t[j] = v[(j + k) & 7];
#pragma unroll
            for (int j = 0; j < 8; j++) v[j] = t[j];
        }
    }
}

// Applies one F_TC op to the tile.  bh/bl: B hi/lo parts in shared memory; aoff: the op's
// 2^k amplitude offsets inside a group (shared memory).
//
// Shared-memory access: lane l of a warp owns group g and visits the 8 amplitudes of each
// chunk starting at (l & 7), so the 32 lanes of a warp touch 8 different offsets at a time
// instead of 32 times the same bank when groups sit 2^k amplitudes apart; a 3-stage select
// network puts the values back in column order for tcgen05.st (and the reverse for D).
// Row tiles [tb, te) of the op (tc_apply below picks the ranges).
__device__ void tc_apply_tiles(float2 *tile, const KOp &op, const float *bh, const float *bl, const uint32_t *aoff,
                               uint32_t tmem, uint64_t *bar, uint32_t &mma_phase, int *abort_flag, int tb,
                               int te) {
    const int k = op.k;
    const int D = 1 << k;             // amplitudes per group
    const int K2 = 2 * D;             // reals per group (GEMM K and N)
    const int RT = te;                // tiles run from tb to te
    const int NT = te - tb;           // row tiles held in TMEM at once
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wg = warp >> 2, wq = warp & 3;
    const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
    const int rsh = lane & 7;
    // TMEM column layout (tile t at column offset (t - tb) * K2 inside each part)
    const uint32_t col_ah = 0u - (uint32_t)(tb * K2), col_al = (uint32_t)((NT - tb) * K2),
                   col_d = (uint32_t)((2 * NT - tb) * K2);
    // work split: with one row tile both warpgroups share it (even / odd column chunks)
    const int t0 = NT >= 2 ? tb + wg : tb, tstep = NT >= 2 ? 2 : 1;
    const int c0 = NT >= 2 ? 0 : wg, cstep = NT >= 2 ? 1 : 2;
    int sorted[8];
    for (int j = 0; j < k; j++) sorted[j] = op.pos[j];
    for (int a = 1; a < k; a++)
        for (int b = a; b > 0 && sorted[b - 1] > sorted[b]; b--) {
            const int t = sorted[b]; sorted[b] = sorted[b - 1]; sorted[b - 1] = t;
        }
    // 1. A operand into TMEM (hi and lo parts)
    for (int t = t0; t < RT; t += tstep) {
        uint32_t base = (uint32_t)(t * 128 + 32 * wq + lane);
        for (int j = 0; j < k; j++) {
            const int b = sorted[j];
            base = ((base >> b) << (b + 1)) | (base & ((1u << b) - 1u));
        }
        for (int c = c0; c < K2 / 16; c += cstep) {
            float2 a[8];
#pragma unroll
            for (int i = 0; i < 8; i++) a[i] = tile[base | aoff[8 * c + ((i + rsh) & 7)]];
            rot8(a, (8 - rsh) & 7);
            uint32_t vh[16], vl[16];
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const uint32_t hr = tf32_rn(a[i].x), hi = tf32_rn(a[i].y);
                vh[2 * i] = hr;
                vh[2 * i + 1] = hi;
                vl[2 * i] = tf32_rn(__fsub_rn(a[i].x, __uint_as_float(hr)));
                vl[2 * i + 1] = tf32_rn(__fsub_rn(a[i].y, __uint_as_float(hi)));
            }
            tc::st16(tmem + lane_off + col_ah + (uint32_t)(t * K2 + 16 * c), vh);
            tc::st16(tmem + lane_off + col_al + (uint32_t)(t * K2 + 16 * c), vl);
        }
    }
    tc::wait_st();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    // 2. MMAs (one thread): D = Ah Bh + Ah Bl + Al Bh, K = 8 per instruction
    if (threadIdx.x == 0) {
        const uint32_t idesc = tc::idesc_tf32(128, K2);
        const uint32_t lbo = 128, sbo = (uint32_t)(K2 / 4) * 128;
        for (int t = tb; t < RT; t++) {
            const uint32_t d = tmem + col_d + (uint32_t)(t * K2);
            for (int s = 0; s < K2 / 8; s++) {
                const uint32_t ah = tmem + col_ah + (uint32_t)(t * K2 + 8 * s);
                const uint32_t al = tmem + col_al + (uint32_t)(t * K2 + 8 * s);
                const uint64_t dbh = tc::sdesc(bh + 64 * s, lbo, sbo);  // 2 core matrices = 256 B per K-step
                const uint64_t dbl = tc::sdesc(bl + 64 * s, lbo, sbo);
                tc::mma_tf32_ta(d, ah, dbh, idesc, s > 0 ? 1u : 0u);
                tc::mma_tf32_ta(d, ah, dbl, idesc, 1u);
                tc::mma_tf32_ta(d, al, dbh, idesc, 1u);
            }
        }
        tc::commit(bar);
    }
    if (!ptx::mbar_wait_bounded(bar, mma_phase, ptx::kWaitLimitNs)) {
        *abort_flag = 1;
        // MMAs may still be in flight: one more bounded wait before TMEM is released
        ptx::mbar_wait_bounded(bar, mma_phase, ptx::kWaitLimitNs);
    }
    mma_phase ^= 1u;
    tc::fence_after();
    // 3. D back into the tile
    for (int t = t0; t < RT; t += tstep) {
        uint32_t base = (uint32_t)(t * 128 + 32 * wq + lane);
        for (int j = 0; j < k; j++) {
            const int b = sorted[j];
            base = ((base >> b) << (b + 1)) | (base & ((1u << b) - 1u));
        }
        for (int c = c0; c < K2 / 16; c += cstep) {
            uint32_t v[16];
            tc::ld16(tmem + lane_off + col_d + (uint32_t)(t * K2 + 16 * c), v);
            tc::wait_ld();
            float2 a[8];
#pragma unroll
            for (int i = 0; i < 8; i++) a[i] = make_float2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
            rot8(a, rsh);
#pragma unroll
            for (int i = 0; i < 8; i++) tile[base | aoff[8 * c + ((i + rsh) & 7)]] = a[i];
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

// Applies one F_TC op: all row tiles of the tile at once (TMEM holds 3 x RT x 2^(k+1)
// columns), or one row tile after the other when seq (3 x 2^(k+1) columns: k <= 5 fits in
// 256 columns, so two CTAs share an SM and one's MMAs overlap the other's gathers).
__device__ void tc_apply(float2 *tile, const KOp &op, const float *bh, const float *bl, const uint32_t *aoff,
                         uint32_t tmem, uint64_t *bar, uint32_t &mma_phase, int m, int *abort_flag, int seq) {
    const int RT = (1 << (m - op.k)) >> 7;  // 128-group row tiles
    if (!seq) {
        tc_apply_tiles(tile, op, bh, bl, aoff, tmem, bar, mma_phase, abort_flag, 0, RT);
        return;
    }
    for (int t = 0; t < RT; t++) {
        tc_apply_tiles(tile, op, bh, bl, aoff, tmem, bar, mma_phase, abort_flag, t, t + 1);
        if (*(volatile int *)abort_flag) return;
    }
}

__global__ void __launch_bounds__(kTcThreads, 2)
k_chunk_tc(float2 *__restrict__ psi, const ChunkArgs a, const KOp *__restrict__ ops, const float *__restrict__ mats,
           const float *__restrict__ bmats, uint32_t b_floats, int b_resident, int seq, int *__restrict__ err) {
    // TMEM columns: seq (blocks of at most 5 qubits, one row tile at a time) fits in 256, so
    // two CTAs share an SM's 512 columns
    const uint32_t tmem_cols = seq ? 256u : kTmemCols;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2 *tile = (float2 *)smem_raw;
    float *bh = (float *)(smem_raw + ((size_t)8 << a.m));
    float *bl = bh + b_floats;
    __shared__ uint64_t bar_load, bar_mma;
    __shared__ uint32_t s_tmem;
    __shared__ int abort_flag;
    __shared__ int s_loaded;
    __shared__ KOp s_op;
    __shared__ float s_m[kMaxOpReals];
    __shared__ uint32_t s_aoff[64];
    const uint32_t nruns = 1u << (a.m - a.c0);
    const uint32_t run_bytes = 8u << a.c0;
    const uint32_t tile_bytes = 8u << a.m;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar_load, 1);
        ptx::mbar_init(&bar_mma, 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
        s_loaded = -1;
    }
    if (threadIdx.x < 32) {
        tc::alloc(&s_tmem, tmem_cols);
        tc::relinquish();
    }
    if (b_resident) {
        // every B operand of the pass stays in shared memory for the whole kernel
        const float4 *src = (const float4 *)bmats;
        float4 *dst = (float4 *)bh;
        for (uint32_t j = threadIdx.x; j < b_floats / 4; j += blockDim.x) dst[j] = src[j];
        ptx::fence_proxy_async_smem();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    uint32_t load_phase = 0, mma_phase = 0;
    for (uint64_t t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        uint64_t base = t << a.c0;
        for (int j = 0; j < a.nlh; j++) {
            const int b = a.lhigh[j];
            base = ((base >> b) << (b + 1)) | (base & ((1ull << b) - 1ull));
        }
        if (threadIdx.x == 0) ptx::mbar_arrive_expect_tx(&bar_load, tile_bytes);
        __syncthreads();
        for (uint32_t r = threadIdx.x; r < nruns; r += blockDim.x) {
            uint64_t off = 0;
            for (int j = 0; j < a.nlh; j++) off |= (uint64_t)((r >> j) & 1u) << a.lhigh[j];
            ptx::bulk_g2s(tile + ((uint64_t)r << a.c0), psi + (base | off), run_bytes, &bar_load);
        }
        if (!ptx::mbar_wait_bounded(&bar_load, load_phase, ptx::kWaitLimitNs)) {
            abort_flag = 1;
            ptx::mbar_wait_bounded(&bar_load, load_phase, ptx::kWaitLimitNs);
        }
        load_phase ^= 1u;
        __syncthreads();
        if (abort_flag) break;
        for (int i = 0; i < a.n_ops; i++) {
            if (threadIdx.x == 0) s_op = ops[i];
            __syncthreads();
            if (s_op.fkind == F_TC) {
                if (!b_resident && s_loaded != i) {
                    const float4 *src = (const float4 *)(bmats + s_op.mat);
                    float4 *dst = (float4 *)bh;
                    const int n4 = s_op.nmat / 4;   // hi then lo, contiguous
                    for (int j = threadIdx.x; j < n4; j += blockDim.x) {
                        const int half = j >= n4 / 2;
                        float4 *d = half ? (float4 *)bl + (j - n4 / 2) : dst + j;
                        *d = src[j];
                    }
                    ptx::fence_proxy_async_smem();  // generic writes -> read by the MMA (async proxy)
                    __syncthreads();
                    if (threadIdx.x == 0) s_loaded = i;
                }
                if (threadIdx.x < (1 << s_op.k)) {
                    uint32_t o = 0;
                    for (int j = 0; j < s_op.k; j++) o |= (uint32_t)((threadIdx.x >> (s_op.k - 1 - j)) & 1) << s_op.pos[j];
                    s_aoff[threadIdx.x] = o;
                }
                __syncthreads();
                const float *obh = b_resident ? bh + s_op.mat : bh;
                const float *obl = b_resident ? obh + s_op.nmat / 2 : bl;
                tc_apply(tile, s_op, obh, obl, s_aoff, tmem, &bar_mma, mma_phase, a.m, &abort_flag, seq);
                if (abort_flag) break;
            } else {
                for (int j = threadIdx.x; j < s_op.nmat; j += blockDim.x) s_m[j] = mats[s_op.mat + j];
                __syncthreads();
                apply_op_smem<float, false>(tile, s_op, s_m, a.m);
                __syncthreads();
            }
        }
        __syncthreads();
        if (abort_flag) break;
        ptx::fence_proxy_async_smem();
        __syncthreads();
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
    if (abort_flag && threadIdx.x == 0) atomicExch(err, QS_ERR_TIMEOUT);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (threadIdx.x < 32) tc::dealloc(tmem, tmem_cols);
}

}  // namespace

bool tc_available(int m, int k) { return k >= 4 && k <= 6 && m >= k + 7 && m <= 13; }

void launch_chunk_pass_tc(DeviceState &st, uint64_t lmask, const std::vector<KOp> &kops,
                          const std::vector<double> &mats, const std::vector<float> &bmats, uint32_t b_floats) {
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
    if (st.dtype != QS_C64) fail(QS_ERR_UNSUPPORTED, "tensor-core blocks run on complex64 states");
    if ((8u << a.c0) % 16 != 0) fail(QS_ERR_INVALID, "chunk runs must be multiples of 16 bytes");
    std::vector<float> tm(std::max<size_t>(mats.size(), 2));
    for (size_t i = 0; i < mats.size(); i++) tm[i] = (float)mats[i];
    const KOp *d_ops = (const KOp *)upload_params(st, kops.data(), kops.size() * sizeof(KOp));
    const float *d_m = (const float *)upload_params(st, tm.data(), tm.size() * sizeof(float));
    const float *d_b = (const float *)upload_params(st, bmats.data(), bmats.size() * sizeof(float));
    // blocks of at most 5 qubits: one row tile at a time in 256 TMEM columns, two CTAs per SM
    int kmax = 0;
    for (const KOp &k : kops)
        if (k.fkind == F_TC) kmax = std::max(kmax, (int)k.k);
    const int seq = kmax <= 5 ? 1 : 0;
    // B operands: all resident if they fit next to the tile, else one op's at a time
    const size_t tile_bytes = (size_t)8 << a.m;
    const size_t all_b = bmats.size() * sizeof(float);
    const size_t per_cta = seq ? 104 * 1024 : 200 * 1024;
    const int resident = tile_bytes + all_b <= per_cta ? 1 : 0;
    const uint32_t bf = resident ? (uint32_t)bmats.size() : b_floats;
    // tile + B.  512 TMEM columns: at least 120 KB, so that one CTA (one TMEM owner) runs per
    // SM; 256 columns: at least 80 KB, so that at most two do
    size_t smem = tile_bytes + (resident ? all_b : 2 * (size_t)b_floats * sizeof(float));
    smem = std::max<size_t>(smem, seq ? 80 * 1024 : 120 * 1024);
    if (seq && smem > 104 * 1024) fail(QS_ERR_INVALID, "tensor-core chunk pass exceeds shared memory");
    if (smem > 220 * 1024) fail(QS_ERR_INVALID, "tensor-core chunk pass exceeds shared memory");
    static bool attr = false;
    if (!attr) {
        QS_CUDA(cudaFuncSetAttribute(k_chunk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
        // the whole unified L1 as shared memory, so that two CTAs of ~100 KB fit on an SM
        QS_CUDA(cudaFuncSetAttribute(k_chunk_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
        attr = true;
    }
    // seq: two CTAs per SM (each holds 256 of the SM's 512 TMEM columns); CTAs share
    // nothing, so a grid larger than what is resident only queues
    const int grid = seq ? (int)std::min<uint64_t>(a.n_tiles, (uint64_t)device_sm_count() * 2)
                         : persistent_grid((const void *)k_chunk_tc, kTcThreads, smem, a.n_tiles);
    k_chunk_tc<<<grid, kTcThreads, smem, st.stream>>>((float2 *)st.psi, a, d_ops, d_m, d_b, bf, resident, seq,
                                                       st.dev_err);
    QS_CUDA(cudaGetLastError());
    count_launch();
}

// Nearest TF32 value of a float (ties to even), as on the device.
static float tf32_round_host(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    b = (b + 0x0FFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

// B = R (2D x 2D real form of the complex D x D block, interleaved re/im ordering) split
// into TF32 hi and lo parts, each stored in the K-major canonical no-swizzle layout:
// element (n, kk) at (n/8)*SBO + (kk/4)*128 + (n%8)*16 + (kk%4)*4 bytes, SBO = (2D/4)*128.
void build_tc_operand(const std::vector<cd> &G, int k, std::vector<float> &out, int &off, int &count) {
    const int D = 1 << k, K2 = 2 * D;
    const size_t nf = (size_t)K2 * K2;
    off = (int)out.size();
    out.resize(out.size() + 2 * nf, 0.0f);
    float *hi = out.data() + off, *lo = hi + nf;
    const size_t sbo_f = (size_t)(K2 / 4) * 32;  // floats per 8-row group
    for (int n = 0; n < K2; n++)
        for (int kk = 0; kk < K2; kk++) {
            const int r = n >> 1, cr = n & 1, s = kk >> 1, cs = kk & 1;
            const cd g = G[(size_t)r * D + s];
            double v;
            if (cr == 0) v = cs == 0 ? g.real() : -g.imag();
            else v = cs == 0 ? g.imag() : g.real();
            const float h = tf32_round_host((float)v);
            const float l = tf32_round_host((float)(v - (double)h));
            const size_t idx = (size_t)(n / 8) * sbo_f + (size_t)(kk / 4) * 32 + (size_t)(n % 8) * 4 + (kk % 4);
            hi[idx] = h;
            lo[idx] = l;
        }
    count = (int)(2 * nf);
}

}  // namespace qs
