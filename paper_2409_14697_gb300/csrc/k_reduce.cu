// K4/K5: reductions and simple state kernels.
//
//  * norm and <Z_q> for every q in one read pass.  <Z_q> = sum_x |a_x|^2 (1 - 2 bit_q(x))
//    = total - 2 S_q with S_q the probability mass on bit_q = 1.  Each block owns a
//    contiguous chunk of 2^cb amplitudes, so every qubit >= cb is constant over the
//    block and only the block total is needed for it; qubits < cb are split into
//    thread bits and loop bits.  Everything is accumulated in FP64 in a fixed order
//    (per-thread loop, fixed butterfly trees, fixed second stage), so results are
//    bitwise reproducible whatever else runs on the GPU.
//  * top-K |a|^2: exact radix select of the K-th largest key (the bit pattern of the
//    non-negative probability, monotone in its value), then a deterministic gather of
//    the elements above it and of the lowest-index ties, then one-block bitonic sort.
//  * |0...0> and scaling.
#include <algorithm>
#include <mutex>

#include "capi_util.h"
#include "qs_internal.h"

namespace qs {
namespace {

constexpr int kMaxLoopBits = 10;

__device__ __forceinline__ double prob(double2 a) {
    return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
}
__device__ __forceinline__ double prob(float2 a) {
    // products of floats are exact in double
    return __dadd_rn(__dmul_rn((double)a.x, (double)a.x), __dmul_rn((double)a.y, (double)a.y));
}

// Butterfly sum over a warp: fixed order, identical result in every lane.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// part[blk*(cb+1) + 0] = block total; part[blk*(cb+1) + 1 + q] = mass with bit q set, q < cb.
template <typename V>
__global__ void __launch_bounds__(256)
k_expz_part(const V *__restrict__ psi, int cb, int tb, int with_bits, double *__restrict__ part) {
    __shared__ double s_tot[256];
    __shared__ double s_j[kMaxLoopBits][256];
    const int T = 1 << tb, t = threadIdx.x;
    const int jb = cb - tb, J = 1 << jb;
    const uint64_t start = (uint64_t)blockIdx.x << cb;
    double tot = 0.0, jacc[kMaxLoopBits];
#pragma unroll
    for (int b = 0; b < kMaxLoopBits; b++) jacc[b] = 0.0;
    for (int j = 0; j < J; j++) {
        const double p = prob(psi[start + ((uint64_t)j << tb) + t]);
        tot += p;
        if (with_bits) {
#pragma unroll
            for (int b = 0; b < kMaxLoopBits; b++)
                if (b < jb && ((j >> b) & 1)) jacc[b] += p;
        }
    }
    s_tot[t] = tot;
    if (with_bits)
        for (int b = 0; b < jb; b++) s_j[b][t] = jacc[b];
    __syncthreads();
    const int n_out = with_bits ? cb + 1 : 1;
    const int warp = t >> 5, lane = t & 31, nw = (T + 31) >> 5;
    for (int r = warp; r < n_out; r += nw) {
        double v = 0.0;
        for (int u = lane; u < T; u += 32) {
            double x;
            if (r == 0) x = s_tot[u];
            else if (r - 1 < tb) x = ((u >> (r - 1)) & 1) ? s_tot[u] : 0.0;
            else x = s_j[r - 1 - tb][u];
            v += x;
        }
        v = T >= 32 ? warp_sum(v) : v;
        if (T < 32) {  // tiny blocks: lane 0 adds the T lanes in order
            v = 0.0;
            if (lane == 0)
                for (int u = 0; u < T; u++) {
                    double x;
                    if (r == 0) x = s_tot[u];
                    else if (r - 1 < tb) x = ((u >> (r - 1)) & 1) ? s_tot[u] : 0.0;
                    else x = s_j[r - 1 - tb][u];
                    v += x;
                }
        }
        if (lane == 0) part[(uint64_t)blockIdx.x * (cb + 1) + r] = v;
    }
}

// out[0] = total, out[1 + q] = <Z_q> for q < n.  One block per output.
__global__ void __launch_bounds__(256)
k_expz_final(const double *__restrict__ part, uint64_t nblk, int cb, int n_out_q,
             double *__restrict__ out) {
    __shared__ double s[256];
    const int o = blockIdx.x;  // 0: total, 1+q: qubit q
    const int q = o - 1;
    double tot = 0.0, v = 0.0;
    for (uint64_t b = threadIdx.x; b < nblk; b += 256) {
        const double bt = part[b * (cb + 1)];
        tot += bt;
        if (q >= 0) {
            if (q < cb) v += part[b * (cb + 1) + 1 + q];
            else if ((b >> (q - cb)) & 1) v += bt;
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
    (void)n_out_q;
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
           int shift, unsigned long long *__restrict__ hist) {
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

__global__ void k_sel_init(SelState *st, unsigned long long K) {
    st->prefix = 0ull;
    st->need = K;
    st->shift = 0;
    st->pad = 0;
}

// Picks the digit holding the need-th largest key among the matching ones.
__global__ void k_sel_pick(SelState *st, unsigned long long *hist, int shift) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
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
            unsigned int *__restrict__ cnt) {
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
__global__ void k_tie_scan(unsigned int *cnt, uint64_t nblk) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
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
         unsigned long long *__restrict__ out_key, unsigned long long *__restrict__ out_idx) {
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
k_topk_sort(const V *__restrict__ psi, unsigned long long *key, unsigned long long *idx, int K,
            int P, unsigned long long *__restrict__ out_idx, double *__restrict__ out_amp) {
    extern __shared__ unsigned long long sm[];
    unsigned long long *sk = sm, *si = sm + P;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        sk[i] = i < K ? key[i] : 0ull;
        si[i] = i < K ? idx[i] : ~0ull;
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

int chunk_bits(int n) { return std::min(n, std::max(12, n - 18)); }

}  // namespace

void launch_set_zero_state(DeviceState &st) {
    const size_t B = st.dtype == QS_C128 ? 16 : 8;
    QS_CUDA(cudaMemsetAsync(st.psi, 0, B << st.n, st.stream));
    k_set_one<<<1, 1, 0, st.stream>>>(st.psi, st.dtype == QS_C128);
    QS_CUDA(cudaGetLastError());
    count_launch();
}

void launch_scale(DeviceState &st, double f) {
    const uint64_t n = 1ull << st.n;
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)device_sm_count() * 8);
    if (st.dtype == QS_C128) k_scale<double2, double><<<grid, 256, 0, st.stream>>>((double2 *)st.psi, n, f);
    else k_scale<float2, float><<<grid, 256, 0, st.stream>>>((float2 *)st.psi, n, (float)f);
    QS_CUDA(cudaGetLastError());
    count_launch();
}

size_t scratch_expz_bytes(int n) {
    const int cb = chunk_bits(n);
    const uint64_t nblk = 1ull << (n - cb);
    return (nblk * (cb + 1) + n + 1) * sizeof(double);
}

// Norm and <Z_q> into out_dev (n + 1 doubles); the partials use st.scratch.
static void expz_launch(DeviceState &st, bool bits, double *out_dev) {
    const int n = st.n;
    const int cb = chunk_bits(n);
    const int tb = std::min(cb, 8);
    const uint64_t nblk = 1ull << (n - cb);
    ensure_scratch(st, scratch_expz_bytes(n));
    double *part = (double *)st.scratch;
    if (st.dtype == QS_C128)
        k_expz_part<double2><<<(unsigned)nblk, 1 << tb, 0, st.stream>>>((const double2 *)st.psi, cb, tb, bits, part);
    else
        k_expz_part<float2><<<(unsigned)nblk, 1 << tb, 0, st.stream>>>((const float2 *)st.psi, cb, tb, bits, part);
    QS_CUDA(cudaGetLastError());
    k_expz_final<<<bits ? n + 1 : 1, 256, 0, st.stream>>>(part, nblk, cb, n, out_dev);
    QS_CUDA(cudaGetLastError());
    count_launch(2);
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
    const int cb = chunk_bits(n);
    const uint64_t nblk = 1ull << (n - cb);
    double *out = (double *)st.scratch + nblk * (cb + 1);
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
    size_t o_sel, o_hist, o_tie, o_gt, o_key, o_idx, o_oidx, o_oamp, total;
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
    L.total = off;
    return L;
}
}  // namespace

size_t scratch_topk_bytes(int n, uint32_t k) { return topk_layout(n, k).total; }

// Launches the whole top-K pipeline; results to idx_dev / amp_dev (device).
void top_k_async(DeviceState &st, uint32_t K, uint64_t *idx_dev, double *amp_dev) {
    const int n = st.n;
    const uint64_t N = 1ull << n;
    if (K == 0) return;
    if (K > N || K > 4096) fail(QS_ERR_INVALID, "top-k: k exceeds min(2^n, 4096)");
    const int cb = std::min(n, 12);
    const uint64_t nblk = N >> cb;
    const TopkLayout TL = topk_layout(n, K);
    const size_t o_sel = TL.o_sel, o_hist = TL.o_hist, o_tie = TL.o_tie, o_gt = TL.o_gt, o_key = TL.o_key,
                 o_idx = TL.o_idx;
    ensure_scratch(st, TL.total);
    char *base = (char *)st.scratch;
    SelState *sel = (SelState *)(base + o_sel);
    unsigned long long *hist = (unsigned long long *)(base + o_hist);
    k_sel_init<<<1, 1, 0, st.stream>>>(sel, (unsigned long long)K);
    count_launch();
    QS_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kBins, st.stream));
    QS_CUDA(cudaMemsetAsync(base + o_gt, 0, sizeof(unsigned int), st.stream));
    const int grid = (int)std::min<uint64_t>((N + 255) / 256, (uint64_t)device_sm_count() * 8);
    // keys are non-negative doubles: bit 63 is always 0, digits cover bits 62..0
    int hi = 64;
    for (int shift = 63 - kDigitBits; hi > 0; shift -= kDigitBits) {
        const int sh = std::max(shift, 0);
        if (st.dtype == QS_C128)
            k_sel_hist<double2><<<grid, 256, 0, st.stream>>>((const double2 *)st.psi, N, sel, hi, sh, hist);
        else
            k_sel_hist<float2><<<grid, 256, 0, st.stream>>>((const float2 *)st.psi, N, sel, hi, sh, hist);
        k_sel_pick<<<1, 1, 0, st.stream>>>(sel, hist, sh);
        count_launch(2);
        hi = sh;
    }
    unsigned int *tie = (unsigned int *)(base + o_tie);
    if (st.dtype == QS_C128)
        k_tie_count<double2><<<(unsigned)nblk, 256, 0, st.stream>>>((const double2 *)st.psi, cb, sel, tie);
    else
        k_tie_count<float2><<<(unsigned)nblk, 256, 0, st.stream>>>((const float2 *)st.psi, cb, sel, tie);
    k_tie_scan<<<1, 1, 0, st.stream>>>(tie, nblk);
    unsigned long long *gkey = (unsigned long long *)(base + o_key), *gidx = (unsigned long long *)(base + o_idx);
    if (st.dtype == QS_C128)
        k_gather<double2><<<(unsigned)nblk, 256, 0, st.stream>>>((const double2 *)st.psi, cb, sel, K, tie,
                                                                   (unsigned int *)(base + o_gt), gkey, gidx);
    else
        k_gather<float2><<<(unsigned)nblk, 256, 0, st.stream>>>((const float2 *)st.psi, cb, sel, K, tie,
                                                                  (unsigned int *)(base + o_gt), gkey, gidx);
    int P = 1;
    while (P < (int)K) P <<= 1;
    P = std::max(P, 2);
    const size_t smem = sizeof(unsigned long long) * 2 * P;
    unsigned long long *oidx = (unsigned long long *)idx_dev;
    double *oamp = amp_dev;
    if (st.dtype == QS_C128) {
        auto kern = k_topk_sort<double2>;
        QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<1, 1024, smem, st.stream>>>((const double2 *)st.psi, gkey, gidx, (int)K, P, oidx, oamp);
    } else {
        auto kern = k_topk_sort<float2>;
        QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<1, 1024, smem, st.stream>>>((const float2 *)st.psi, gkey, gidx, (int)K, P, oidx, oamp);
    }
    QS_CUDA(cudaGetLastError());
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
constexpr size_t kNoAllocScratchDoubles = ((size_t)1 << kNoAllocMaxBlockBits) * 19 + 64;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[64] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
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
    const int tb = std::min(cb, 8);
    const uint64_t nblk = 1ull << (n - cb);
    const size_t part_elems = nblk * (cb + 1);
    if (part_elems + n + 1 > kNoAllocScratchDoubles) fail(QS_ERR_INVALID, "static scratch too small");
    double *part = noalloc_scratch();
    double *out = part + part_elems;
    cudaStream_t st = (cudaStream_t)stream;
    // every partial the second stage reads is written by the first: nothing to clear
    if (dt == QS_C128)
        k_expz_part<double2><<<(unsigned)nblk, 1 << tb, 0, st>>>((const double2 *)dev_psi, cb, tb, 1, part);
    else
        k_expz_part<float2><<<(unsigned)nblk, 1 << tb, 0, st>>>((const float2 *)dev_psi, cb, tb, 1, part);
    QS_CUDA(cudaGetLastError());
    k_expz_final<<<n + 1, 256, 0, st>>>(part, nblk, cb, n, out);
    QS_CUDA(cudaGetLastError());
    count_launch(2);
    double h[kNoAllocMaxQubits + 1];
    QS_CUDA(cudaMemcpyAsync(h, out, sizeof(double) * (n + 1), cudaMemcpyDeviceToHost, st));
    QS_CUDA(cudaStreamSynchronize(st));
    if (out_norm) *out_norm = h[0];
    if (out_expz)
        for (int q = 0; q < n; q++) out_expz[q] = h[1 + q];
    QS_API_END
}

