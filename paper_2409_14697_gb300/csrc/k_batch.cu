// K6: many independent circuits in ONE persistent launch (captured in a CUDA graph).
//
// Every circuit is planned on the host into passes exactly like a single state
// (plan.cpp: local qubits, ops fused inside the pass, tile-local positions).  A pass of
// circuit c is split into tiles; all tiles of all passes form one global work list,
// ordered level by level (every circuit's first pass, then every second pass, ...).
// Persistent CTAs take work items from an atomic counter.  A circuit small enough to fit
// one tile (2^n <= 2^m) is a single item: its state is built as |0...0> in shared memory,
// all of its gates run there, and it is written to HBM once.  A later pass of a larger
// circuit waits (bounded) until every tile of the circuit's previous pass has been
// written; items are handed out in dependency order to CTAs that are already running,
// so the wait always ends.  Tiles move by TMA bulk copies as in the chunk kernel.
#include <algorithm>
#include <cstring>

#include "batch.h"
#include "chunk.h"
#include "kgeom.h"
#include "plan.h"
#include "ptx.cuh"
#include "tile_ops.cuh"

namespace qs {
namespace {

constexpr int kBatchThreads = kTileThreads;
// Largest pass program (ops + reals) staged in shared memory per work item; two CTAs per SM
// must still fit next to their 64 KiB tiles.
constexpr size_t kBatchProgMax = 36 * 1024;

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
using ptx::globaltimer_ns;

template <typename T>
__global__ void __launch_bounds__(kBatchThreads, 2)
k_batch(typename C2T<T>::type *__restrict__ states, const BatchPass *__restrict__ passes, int n_passes,
        uint64_t total_items, const KOp *__restrict__ ops, const T *__restrict__ mats,
        unsigned long long *__restrict__ counter, unsigned int *__restrict__ done, int *__restrict__ err,
        int *__restrict__ abort_all, long long wait_limit_ns, uint32_t prog_off) {
    using V = typename C2T<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V *tile = (V *)smem_raw;
    __shared__ uint64_t bar;
    __shared__ BatchPass s_pass;
    __shared__ unsigned long long s_w;
    __shared__ int s_stop;
    __shared__ KOp s_op;
    __shared__ T s_m[kMaxOpReals];
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            s_stop = 0;
            const unsigned long long w = atomicAdd(counter, 1ull);
            s_w = w;
            if (w >= total_items || *(volatile int *)abort_all) {
                s_stop = 1;
            } else {
                int lo = 0, hi = n_passes - 1;  // last pass with tile_start <= w
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (passes[mid].tile_start <= w) lo = mid;
                    else hi = mid - 1;
                }
                s_pass = passes[lo];
                const int dep = s_pass.dep;
                if (dep >= 0) {
                    const unsigned int need = s_pass.dep_need;
                    const uint64_t t0 = globaltimer_ns();
                    while (ld_acquire(done + dep) < need) {
                        if (*(volatile int *)abort_all) {
                            s_stop = 1;
                            break;
                        }
                        if ((long long)(globaltimer_ns() - t0) > wait_limit_ns) {
                            atomicExch(err, QS_ERR_TIMEOUT);
                            atomicExch(abort_all, 1);
                            s_stop = 1;
                            break;
                        }
                        __nanosleep(256);
                    }
                }
            }
        }
        __syncthreads();
        if (s_stop) break;
        const BatchPass &bp = s_pass;
        const uint64_t t = s_w - bp.tile_start;
        uint32_t nruns = 1u << (bp.m - bp.c0);
        uint32_t run_bytes = (uint32_t)sizeof(V) << bp.c0;
        const uint32_t tile_amps = 1u << bp.m;
        uint64_t base = t << bp.c0;
        for (int j = 0; j < bp.nlh; j++) {
            const int b = bp.lhigh[j];
            base = ((base >> b) << (b + 1)) | (base & ((1ull << b) - 1ull));
        }
        V *psi = states + bp.state_off;
        if (bp.init_zero) {
            for (uint32_t x = threadIdx.x; x < tile_amps; x += blockDim.x) {
                V z;
                z.x = (base == 0 && x == 0) ? (T)1 : (T)0;
                z.y = (T)0;
                tile[x] = z;
            }
            __syncthreads();
        } else {
            fence_proxy_async_global();  // order the acquire above before TMA reads
            if (threadIdx.x == 0) ptx::mbar_arrive_expect_tx(&bar, (uint32_t)sizeof(V) << bp.m);
            __syncthreads();
            for (uint32_t r = threadIdx.x; r < nruns; r += blockDim.x) {
                uint64_t off = 0;
                for (int j = 0; j < bp.nlh; j++) off |= (uint64_t)((r >> j) & 1u) << bp.lhigh[j];
                ptx::bulk_g2s(tile + ((uint64_t)r << bp.c0), psi + (base | off), run_bytes, &bar);
            }
            const uint64_t t0 = globaltimer_ns();
            bool ok = true;
            while (!ptx::mbar_try_wait(&bar, phase)) {
                if ((long long)(globaltimer_ns() - t0) > wait_limit_ns) {
                    ok = false;
                    break;
                }
            }
            if (!ok) {
                atomicExch(err, QS_ERR_TIMEOUT);
                atomicExch(abort_all, 1);
                // give copies still in flight one more bounded wait before leaving
                const uint64_t t1 = globaltimer_ns();
                while (!ptx::mbar_try_wait(&bar, phase) && (long long)(globaltimer_ns() - t1) < wait_limit_ns) {
                }
            }
            phase ^= 1u;
            __syncthreads();
            if (*(volatile int *)abort_all) break;
        }
        // one call site of the op code (register phases are large); a staged pass has its ops
        // and reals copied once per work item, then needs one barrier per op
        KOp *st_ops = (KOp *)(smem_raw + prog_off);
        T *st_m = (T *)(smem_raw + prog_off + (size_t)bp.n_ops * sizeof(KOp));
        if (bp.staged) {
            const uint32_t *src = (const uint32_t *)(ops + bp.ops_off);
            uint32_t *dst = (uint32_t *)st_ops;
            const uint32_t nw = (uint32_t)bp.n_ops * (uint32_t)(sizeof(KOp) / 4);
            for (uint32_t j = threadIdx.x; j < nw; j += blockDim.x) dst[j] = src[j];
            for (uint32_t j = threadIdx.x; j < bp.n_reals; j += blockDim.x) st_m[j] = mats[bp.mats_off + j];
            __syncthreads();
        }
        for (int i = 0; i < bp.n_ops; i++) {
            const KOp *op;
            const T *om;
            if (bp.staged) {
                op = st_ops + i;
                om = st_m + op->mat;
            } else {
                if (threadIdx.x == 0) s_op = ops[bp.ops_off + i];
                __syncthreads();
                for (int j = threadIdx.x; j < s_op.nmat; j += blockDim.x) s_m[j] = mats[bp.mats_off + s_op.mat + j];
                __syncthreads();
                op = &s_op;
                om = s_m;
            }
            apply_op_smem<T>(tile, *op, om, bp.m);
            __syncthreads();
        }
        ptx::fence_proxy_async_smem();
        __syncthreads();
        // the write-back addresses are rebuilt from shared memory instead of being kept live
        // through the ops (register pressure of the complex64 register phases)
        asm volatile("" ::: "memory");
        base = (s_w - bp.tile_start) << bp.c0;
        for (int j = 0; j < bp.nlh; j++) {
            const int b = bp.lhigh[j];
            base = ((base >> b) << (b + 1)) | (base & ((1ull << b) - 1ull));
        }
        psi = states + bp.state_off;
        nruns = 1u << (bp.m - bp.c0);
        run_bytes = (uint32_t)sizeof(V) << bp.c0;
        for (uint32_t r = threadIdx.x; r < nruns; r += blockDim.x) {
            uint64_t off = 0;
            for (int j = 0; j < bp.nlh; j++) off |= (uint64_t)((r >> j) & 1u) << bp.lhigh[j];
            ptx::bulk_s2g(psi + (base | off), tile + ((uint64_t)r << bp.c0), run_bytes);
        }
        ptx::bulk_commit();
        ptx::bulk_wait_all();       // writes complete before the tile is reported done
        fence_proxy_async_global();
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) red_release_add(done + s_pass.self, 1u);
    }
    ptx::bulk_wait_all();
}

}  // namespace

template <typename T>
void launch_batch_kernel(Batch &b) {
    using V = typename C2T<T>::type;
    auto kern = k_batch<T>;
    static bool attr_set[2] = {false, false};
    if (!attr_set[sizeof(T) == 8]) {
        QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        // the whole unified L1 as shared memory: two CTAs of up to ~104 KB per SM
        QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
        attr_set[sizeof(T) == 8] = true;
    }
    const size_t tile_bytes = sizeof(V) << b.max_m;
    const size_t smem = tile_bytes + b.prog_bytes;
    b.grid = persistent_grid((const void *)kern, kBatchThreads, smem, b.total_items);
    QS_CUDA(cudaMemsetAsync(b.d_counter, 0, sizeof(unsigned long long), b.stream));
    QS_CUDA(cudaMemsetAsync(b.d_done, 0, sizeof(unsigned int) * b.passes.size(), b.stream));
    kern<<<b.grid, kBatchThreads, smem, b.stream>>>((V *)b.d_states, b.d_passes, (int)b.passes.size(),
                                                   b.total_items, b.d_ops, (const T *)b.d_mats, b.d_counter,
                                                   b.d_done, b.d_err, b.d_abort, b.wait_limit_ns,
                                                   (uint32_t)tile_bytes);
    QS_CUDA(cudaGetLastError());
    count_launch();
}

void batch_build(Batch &b, const std::vector<std::vector<Op>> &circ_ops, const std::vector<int> &nq,
                 const qs_options &o) {
    const bool c128 = b.dtype == QS_C128;
    const size_t B = c128 ? 16 : 8;
    const int m_max = o.chunk_m > 0 ? o.chunk_m : (c128 ? 12 : 13);
    b.max_m = 0;
    b.prog_bytes = 0;
    // per-circuit planning
    struct CP { std::vector<Pass> plan; std::vector<std::vector<KOp>> kops; std::vector<std::vector<double>> mats; std::vector<uint64_t> lm; };
    std::vector<CP> cps(circ_ops.size());
    uint64_t state_off = 0;
    b.state_off.resize(circ_ops.size());
    int max_level = 0;
    for (size_t c = 0; c < circ_ops.size(); c++) {
        const int n = nq[c];
        DeviceState d;
        d.n = n;
        d.dtype = b.dtype;
        d.reg_phases = (o.flags & QS_OPT_NO_REG_PHASES) == 0;
        qs_options oc = o;
        oc.chunk_m = std::min(m_max, n);
        PlanParams pp = plan_params(d, oc);
        pp.hi_diag = false;  // the batched kernel applies ops on local qubits only
        pp.c = std::min(pp.c, std::max(1, pp.m - 2));
        if ((B << pp.c) < 16) pp.c = c128 ? 1 : 1;
        CP &cp = cps[c];
        cp.plan = make_plan(circ_ops[c], n, pp);
        for (Pass &p : cp.plan) {
            uint64_t L = p.lmask;
            if (L == 0 || p.stream) {
                // single-op passes still run as tiles here
                L = (1ull << pp.c) - 1ull;
                for (int i : p.ops) L |= circ_ops[c][i].qmask();
                for (int bit = 0; bit < n && __builtin_popcountll(L) < pp.m; bit++) L |= 1ull << bit;
            }
            if (__builtin_popcountll(L) > pp.m) fail(QS_ERR_UNSUPPORTED, "batched op wider than the tile");
            for (int i : p.ops)
                if (circ_ops[c][i].kind == K_DENSE && circ_ops[c][i].k > 4)
                    fail(QS_ERR_UNSUPPORTED, "batched circuits take dense blocks of at most 4 qubits");
            std::vector<Op> pops;
            for (int i : p.ops) pops.push_back(circ_ops[c][i]);
            const std::vector<Op> fused = fuse_ops(std::move(pops), pp.fuse_k, pp.sweep_flops);
            int pos[64] = {0};
            int r = 0;
            for (int bit = 0; bit < n; bit++)
                if ((L >> bit) & 1ull) pos[bit] = r++;
            std::vector<KOp> ko;
            std::vector<double> mt;
            const int m = __builtin_popcountll(L);
            if (!c128 && d.reg_phases && rphase_applicable(m, kTileThreadBits)) {
                ko = build_register_phases(fused, pos, m, kTileThreadBits, mt);
            } else {
                for (const Op &op : fused) ko.push_back(make_kop(op, pos, mt));
            }
            cp.kops.push_back(std::move(ko));
            cp.mats.push_back(std::move(mt));
            cp.lm.push_back(L);
            b.max_m = std::max(b.max_m, __builtin_popcountll(L));
        }
        max_level = std::max(max_level, (int)cp.plan.size());
        b.state_off[c] = state_off;
        state_off += 1ull << n;
        // keep every state 256-byte aligned
        const uint64_t align = 256 / B;
        state_off = (state_off + align - 1) / align * align;
    }
    b.state_elems = state_off;
    // global pass order: level by level
    std::vector<double> all_mats;
    std::vector<KOp> all_ops;
    b.passes.clear();
    std::vector<int> last_pass(circ_ops.size(), -1);
    uint64_t items = 0;
    b.total_passes_per_circuit.assign(circ_ops.size(), 0);
    for (int lvl = 0; lvl < max_level; lvl++) {
        for (size_t c = 0; c < circ_ops.size(); c++) {
            if (lvl >= (int)cps[c].plan.size()) continue;
            const uint64_t L = cps[c].lm[lvl];
            const int n = nq[c];
            BatchPass bp{};
            bp.circuit = (int32_t)c;
            bp.self = (int32_t)b.passes.size();
            bp.m = __builtin_popcountll(L);
            bp.c0 = 0;
            while (bp.c0 < n && ((L >> bp.c0) & 1ull)) bp.c0++;
            bp.nlh = 0;
            for (int bit = bp.c0; bit < n; bit++)
                if ((L >> bit) & 1ull) bp.lhigh[bp.nlh++] = bit;
            bp.n_ops = (int32_t)cps[c].kops[lvl].size();
            bp.init_zero = lvl == 0 ? 1 : 0;
            bp.dep = last_pass[c];
            bp.dep_need = bp.dep >= 0 ? b.passes[bp.dep].n_tiles : 0;
            bp.n_tiles = (uint32_t)(1ull << (n - bp.m));
            bp.state_off = b.state_off[c];
            bp.tile_start = items;
            bp.ops_off = all_ops.size();
            bp.mats_off = all_mats.size();
            bp.n_reals = (uint32_t)cps[c].mats[lvl].size();
            {
                const size_t prog = (size_t)bp.n_ops * sizeof(KOp) + (size_t)bp.n_reals * B / 2;
                bp.staged = prog <= kBatchProgMax ? 1 : 0;
                if (bp.staged) b.prog_bytes = std::max(b.prog_bytes, (prog + 15) / 16 * 16);
            }
            if ((B << bp.c0) % 16 != 0) fail(QS_ERR_UNSUPPORTED, "batched tile runs below 16 bytes");
            items += bp.n_tiles;
            all_ops.insert(all_ops.end(), cps[c].kops[lvl].begin(), cps[c].kops[lvl].end());
            all_mats.insert(all_mats.end(), cps[c].mats[lvl].begin(), cps[c].mats[lvl].end());
            last_pass[c] = bp.self;
            b.passes.push_back(bp);
            b.total_passes_per_circuit[c]++;
        }
    }
    b.total_items = items;
    // test hook: make the first dependent pass wait on a pass that never completes
    if (o.reserved[1] == 1) {
        for (BatchPass &bp : b.passes)
            if (bp.dep >= 0) {
                bp.dep = (int32_t)b.passes.size();  // an extra counter that nothing increments
                bp.dep_need = 1;
                break;
            }
    }
    // device buffers
    const size_t mat_elem = c128 ? 8 : 4;
    std::vector<char> mats_t(all_mats.size() * mat_elem + 16);
    for (size_t i = 0; i < all_mats.size(); i++) {
        if (c128) ((double *)mats_t.data())[i] = all_mats[i];
        else ((float *)mats_t.data())[i] = (float)all_mats[i];
    }
    QS_CUDA(cudaMalloc(&b.d_states, b.state_elems * B));
    QS_CUDA(cudaMalloc(&b.d_passes, sizeof(BatchPass) * std::max<size_t>(b.passes.size(), 1)));
    QS_CUDA(cudaMalloc(&b.d_ops, sizeof(KOp) * std::max<size_t>(all_ops.size(), 1)));
    QS_CUDA(cudaMalloc(&b.d_mats, mats_t.size()));
    QS_CUDA(cudaMalloc(&b.d_counter, sizeof(unsigned long long)));
    QS_CUDA(cudaMalloc(&b.d_done, sizeof(unsigned int) * (b.passes.size() + 1)));
    QS_CUDA(cudaMalloc(&b.d_err, sizeof(int)));
    QS_CUDA(cudaMalloc(&b.d_abort, sizeof(int)));
    QS_CUDA(cudaMemcpy(b.d_passes, b.passes.data(), sizeof(BatchPass) * b.passes.size(), cudaMemcpyHostToDevice));
    if (!all_ops.empty())
        QS_CUDA(cudaMemcpy(b.d_ops, all_ops.data(), sizeof(KOp) * all_ops.size(), cudaMemcpyHostToDevice));
    QS_CUDA(cudaMemcpy(b.d_mats, mats_t.data(), mats_t.size(), cudaMemcpyHostToDevice));
    QS_CUDA(cudaMemset(b.d_err, 0, sizeof(int)));
    QS_CUDA(cudaMemset(b.d_abort, 0, sizeof(int)));
    QS_CUDA(cudaMemset(b.d_done, 0, sizeof(unsigned int) * (b.passes.size() + 1)));
    b.wait_limit_ns = (o.reserved[0] > 0 ? (long long)o.reserved[0] : 2000000ll) * 1000ll;
}

void batch_capture(Batch &b) {
    // one graph: reset counters + the persistent kernel
    cudaStream_t cap;
    QS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t keep = b.stream;
    b.stream = cap;
    QS_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    try {
        if (b.dtype == QS_C128) launch_batch_kernel<double>(b);
        else launch_batch_kernel<float>(b);
    } catch (...) {
        cudaGraph_t g;
        cudaStreamEndCapture(cap, &g);
        if (g) cudaGraphDestroy(g);
        b.stream = keep;
        cudaStreamDestroy(cap);
        throw;
    }
    cudaGraph_t g = nullptr;
    QS_CUDA(cudaStreamEndCapture(cap, &g));
    b.stream = keep;
    QS_CUDA(cudaStreamDestroy(cap));
    QS_CUDA(cudaGraphInstantiate(&b.exec, g, 0));
    QS_CUDA(cudaGraphDestroy(g));
}

}  // namespace qs
