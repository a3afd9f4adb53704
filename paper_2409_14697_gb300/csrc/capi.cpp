// C interface (include/qs.h): state handles, the circuit executor, amplitude I/O and
// reductions.  Every C entry point catches qs::Error and returns its code.
#include <atomic>
#include <cstring>
#include <mutex>

#include "capi_util.h"
#include "chunk.h"
#include "plan.h"
#include "qs_internal.h"

struct qs_state {
    qs::DeviceState d;
    bool owns_memory = true;
    bool owns_stream = true;
    qs_stats stats{};
};

namespace qs {

thread_local std::string g_last_error;
namespace {
std::atomic<uint64_t> g_launches{0};
}  // namespace

void fail(int code, const std::string &msg) { throw Error{code, msg}; }

void cuda_check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        const int code = (e == cudaErrorMemoryAllocation) ? QS_ERR_NOMEM : QS_ERR_CUDA;
        fail(code, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int device_sm_count() {
    int dev = 0;
    QS_CUDA(cudaGetDevice(&dev));
    static std::mutex mu;
    static int cache[64] = {0};
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && cache[dev]) return cache[dev];
    int sms = 0;
    QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dev < 64) cache[dev] = sms;
    return sms;
}

// Device buffers a state grows while it runs (scratch, parameter arenas, the booster's
// sub-states) are stream-ordered allocations on the state's stream: growing one never waits
// for the whole device (cudaFree does), which would stall a serving worker behind every
// request in flight.
void ensure_scratch(DeviceState &st, size_t bytes) {
    if (st.scratch_bytes >= bytes) return;
    if (st.scratch) {
        QS_CUDA(cudaFreeAsync(st.scratch, st.stream));
        st.scratch = nullptr;
        st.scratch_bytes = 0;
    }
    const size_t cap = std::max<size_t>(bytes, 1 << 20);
    QS_CUDA(cudaMallocAsync(&st.scratch, cap, st.stream));
    st.scratch_bytes = cap;
}

// Parameter arenas: a ring of kArenas used in turn by successive qs_apply_circuit calls.
// Before an arena is reused, the event recorded after its last copy is waited on, so the
// pinned staging memory is never rewritten while a copy from it may still be pending.
void arena_begin(DeviceState &st) {
    st.arena_cur = (st.arena_cur + 1) % kArenas;
    st.arena_used = 0;
    const int c = st.arena_cur;
    if (st.arena_ev[c]) QS_CUDA(cudaEventSynchronize(st.arena_ev[c]));
    // buffers this arena outgrew during its last use are idle now; the page-locked ones are
    // kept until the state is freed (cudaFreeHost waits for the whole device)
    for (auto &r : st.arena_retired[c]) {
        if (r.first) QS_CUDA(cudaFreeAsync(r.first, st.stream));
        if (r.second) st.pinned_retired.push_back(r.second);
    }
    st.arena_retired[c].clear();
}

void arena_end(DeviceState &st) {
    if (!st.arena_ev[st.arena_cur])
        QS_CUDA(cudaEventCreateWithFlags(&st.arena_ev[st.arena_cur], cudaEventDisableTiming));
    QS_CUDA(cudaEventRecord(st.arena_ev[st.arena_cur], st.stream));
}

void arena_reserve(DeviceState &st, size_t bytes) {
    for (int c = 0; c < kArenas; c++) {
        if (st.arena_cap[c] >= bytes) continue;
        if (st.arena_ev[c]) QS_CUDA(cudaEventSynchronize(st.arena_ev[c]));
        if (st.arena_dev[c]) QS_CUDA(cudaFreeAsync(st.arena_dev[c], st.stream));
        if (st.arena_host[c]) st.pinned_retired.push_back(st.arena_host[c]);
        st.arena_dev[c] = st.arena_host[c] = nullptr;
        st.arena_cap[c] = 0;
        QS_CUDA(cudaMallocAsync(&st.arena_dev[c], bytes, st.stream));
        QS_CUDA(cudaMallocHost(&st.arena_host[c], bytes));
        st.arena_cap[c] = bytes;
    }
}

void *upload_params(DeviceState &st, const void *host, size_t bytes) {
    const int c = st.arena_cur;
    const size_t need = ((st.arena_used + 255) & ~size_t(255)) + bytes;
    if (need > st.arena_cap[c]) {
        // grow: earlier uploads of this call (and queued copies from the pinned staging)
        // still refer to the old buffers, so they are retired, not freed; arena_begin frees
        // them once this arena's event shows that nothing uses them
        st.arena_retired[c].push_back({st.arena_dev[c], st.arena_host[c]});
        st.arena_dev[c] = st.arena_host[c] = nullptr;
        const size_t cap = std::max<size_t>(need * 2, 1 << 16);
        QS_CUDA(cudaMallocAsync(&st.arena_dev[c], cap, st.stream));
        QS_CUDA(cudaMallocHost(&st.arena_host[c], cap));
        st.arena_cap[c] = cap;
        st.arena_used = 0;
    }
    const size_t off = (st.arena_used + 255) & ~size_t(255);
    std::memcpy((char *)st.arena_host[c] + off, host, bytes);
    void *dst = (char *)st.arena_dev[c] + off;
    QS_CUDA(cudaMemcpyAsync(dst, (char *)st.arena_host[c] + off, bytes, cudaMemcpyHostToDevice, st.stream));
    st.arena_used = off + bytes;
    return dst;
}

// Waits for the state's stream, then reports (and clears) a device-side timeout.
void sync_and_check(DeviceState &d) {
    QS_CUDA(cudaStreamSynchronize(d.stream));
    if (!d.dev_err) return;
    int e = 0;
    QS_CUDA(cudaMemcpy(&e, d.dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
        QS_CUDA(cudaMemset(d.dev_err, 0, sizeof(int)));
        fail(e, "a bounded device-side wait gave up (kernel returned early)");
    }
}

static size_t amp_bytes(int dtype) { return dtype == QS_C128 ? 16 : 8; }

static void destroy_state(qs_state *s) {
    DeviceState &d = s->d;
    free_device_state(d);
    if (s->owns_memory && d.psi) cudaFree(d.psi);
    if (s->owns_stream && d.stream) cudaStreamDestroy(d.stream);
    delete s;
}

// Runs the executor for one circuit (validated, lowered) on d.stream.
void run_circuit(DeviceState &d, const std::vector<Op> &ops, const qs_options &o, qs_stats &st) {
    st = qs_stats{};
    st.gates_in = (int64_t)ops.size();
    if (o.precision != QS_PREC_DEFAULT && o.precision != QS_PREC_FP64 && o.precision != QS_PREC_DF32 &&
        o.precision != QS_PREC_IX64)
        fail(QS_ERR_INVALID, "unknown precision mode");
    d.prec = o.precision == QS_PREC_DF32 ? QS_PREC_DF32 : QS_PREC_FP64;
    d.ix = o.precision == QS_PREC_IX64 || o.precision == QS_PREC_DEFAULT;
    d.reg_phases = (o.flags & QS_OPT_NO_REG_PHASES) == 0;
    const uint64_t l0 = g_launches.load();
    arena_begin(d);
    const int mode = o.mode;
    try {
        if (mode == QS_MODE_GATE) {
            std::vector<Op> gops = fold_global_phases(ops);
            if (d.dtype == QS_C128 && d.prec == QS_PREC_FP64) defer_hadamard_scale(gops);
            for (const Op &op : gops) {
                launch_stream_op(d, op);
                st.passes++;
                st.bytes += stream_bytes(op, d.n, d.dtype);
            }
            st.ops_after_fuse = (int64_t)ops.size();
        } else if (mode == QS_MODE_FUSED) {
            const int k = o.fuse_k > 0 ? o.fuse_k : 3;
            const std::vector<Op> fused = fuse_ops(ops, std::min(k, 6));
            const int m_tc = std::min(d.n, 13);
            for (const Op &op : fused) {
                if (d.dtype == QS_C64 && op.kind == K_DENSE && tc_available(m_tc, op.k)) {
                    // one full pass per block on the tensor cores: local qubits = the
                    // block's qubits plus the lowest others up to 2^13 amplitudes
                    uint64_t L = op.qmask();
                    for (int b = 0; b < d.n && __builtin_popcountll(L) < m_tc; b++) L |= 1ull << b;
                    st.tile_sweeps += launch_pass_ops(d, L, {op}, true, &st);
                    st.bytes += 2.0 * 8.0 * (double)(1ull << d.n);
                } else {
                    launch_stream_op(d, op);
                    st.bytes += stream_bytes(op, d.n, d.dtype);
                }
                st.passes++;
            }
            st.ops_after_fuse = (int64_t)fused.size();
        } else if (mode == QS_MODE_AUTO || mode == QS_MODE_CHUNK) {
            run_planned(d, ops, o, st);
        } else {
            fail(QS_ERR_INVALID, "unknown mode");
        }
    } catch (...) {
        arena_end(d);
        d.known_zero = false;
        throw;
    }
    arena_end(d);
    if (!ops.empty()) d.known_zero = false;
    st.launches = (int64_t)(g_launches.load() - l0);
}

void free_device_state(DeviceState &d) {
    if (d.stream) cudaStreamSynchronize(d.stream);
    tpb_free(d);
    for (int c = 0; c < kArenas; c++) {
        if (d.arena_dev[c]) cudaFreeAsync(d.arena_dev[c], d.stream);
        if (d.arena_host[c]) cudaFreeHost(d.arena_host[c]);
        for (auto &r : d.arena_retired[c]) {
            if (r.first) cudaFreeAsync(r.first, d.stream);
            if (r.second) cudaFreeHost(r.second);
        }
        d.arena_retired[c].clear();
        if (d.arena_ev[c]) cudaEventDestroy(d.arena_ev[c]);
        d.arena_dev[c] = d.arena_host[c] = nullptr;
        d.arena_ev[c] = nullptr;
        d.arena_cap[c] = 0;
    }
    for (void *p : d.pinned_retired) cudaFreeHost(p);
    d.pinned_retired.clear();
    if (d.scratch) cudaFreeAsync(d.scratch, d.stream);
    if (d.dev_err) cudaFree(d.dev_err);
    if (d.dev_norms) cudaFree(d.dev_norms);
    d.dev_norms = nullptr;
    d.scratch = nullptr;
    d.scratch_bytes = 0;
    d.dev_err = nullptr;
}

static void execute(qs_state *s, const std::vector<Op> &ops, const qs_options &o) {
    run_circuit(s->d, ops, o, s->stats);
}

}  // namespace qs

using namespace qs;
extern "C" {

const char *qs_last_error(void) { return qs::g_last_error.c_str(); }

uint64_t qs_launch_count(void) { return qs::g_launches.load(); }

int qs_version(int32_t *abi, int32_t *device_count) {
    QS_API_BEGIN
    if (abi) *abi = QS_ABI_VERSION;
    if (device_count) {
        int c = 0;
        if (cudaGetDeviceCount(&c) != cudaSuccess) c = 0;
        *device_count = c;
    }
    QS_API_END
}

static void check_new(int n, qs_dtype dt, qs_state **out) {
    if (!out) fail(QS_ERR_INVALID, "out is NULL");
    if (n < 1 || n > QS_MAX_QUBITS) fail(QS_ERR_INVALID, "n_qubits out of range");
    if (dt != QS_C64 && dt != QS_C128) fail(QS_ERR_INVALID, "unknown dtype");
}

int qs_create(int n_qubits, qs_dtype dt, qs_state **out) {
    QS_API_BEGIN
    check_new(n_qubits, dt, out);
    *out = nullptr;
    qs_state *s = new qs_state();
    s->d.n = n_qubits;
    s->d.dtype = dt;
    try {
        QS_CUDA(cudaStreamCreateWithFlags(&s->d.stream, cudaStreamNonBlocking));
        const size_t bytes = amp_bytes(dt) << n_qubits;
        cudaError_t e = cudaMalloc(&s->d.psi, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->d.psi = nullptr;
            fail(QS_ERR_NOMEM, "cannot allocate " + std::to_string(bytes) + " bytes of device memory");
        }
        QS_CUDA(cudaMalloc(&s->d.dev_err, sizeof(int)));
        QS_CUDA(cudaMemsetAsync(s->d.dev_err, 0, sizeof(int), s->d.stream));
        launch_set_zero_state(s->d);
        QS_CUDA(cudaStreamSynchronize(s->d.stream));
    } catch (...) {
        destroy_state(s);
        throw;
    }
    *out = s;
    QS_API_END
}

int qs_create_on(int n_qubits, qs_dtype dt, void *dev_ptr, uint64_t bytes, void *stream,
                 qs_state **out) {
    QS_API_BEGIN
    check_new(n_qubits, dt, out);
    if (!dev_ptr) fail(QS_ERR_INVALID, "dev_ptr is NULL");
    if (((uintptr_t)dev_ptr & 255) != 0) fail(QS_ERR_INVALID, "dev_ptr must be 256-byte aligned");
    if (bytes < (amp_bytes(dt) << n_qubits)) fail(QS_ERR_INVALID, "buffer too small for the state");
    qs_state *s = new qs_state();
    s->d.n = n_qubits;
    s->d.dtype = dt;
    s->d.psi = dev_ptr;
    s->d.stream = (cudaStream_t)stream;
    s->owns_memory = false;
    s->owns_stream = false;
    try {
        QS_CUDA(cudaMalloc(&s->d.dev_err, sizeof(int)));
        QS_CUDA(cudaMemset(s->d.dev_err, 0, sizeof(int)));
    } catch (...) {
        destroy_state(s);
        throw;
    }
    *out = s;
    QS_API_END
}

int qs_destroy(qs_state *s) {
    QS_API_BEGIN
    if (!s) fail(QS_ERR_INVALID, "state is NULL");
    destroy_state(s);
    QS_API_END
}

int qs_set_stream(qs_state *s, void *stream) {
    QS_API_BEGIN
    if (!s) fail(QS_ERR_INVALID, "state is NULL");
    QS_CUDA(cudaStreamSynchronize(s->d.stream));
    if (s->owns_stream && s->d.stream) QS_CUDA(cudaStreamDestroy(s->d.stream));
    s->d.stream = (cudaStream_t)stream;
    s->owns_stream = false;
    QS_API_END
}

int qs_synchronize(qs_state *s) {
    QS_API_BEGIN
    if (!s) fail(QS_ERR_INVALID, "state is NULL");
    sync_and_check(s->d);
    QS_API_END
}

int qs_reset(qs_state *s) {
    QS_API_BEGIN
    if (!s) fail(QS_ERR_INVALID, "state is NULL");
    launch_set_zero_state(s->d);
    QS_API_END
}

int qs_info(const qs_state *s, int32_t *n_qubits, int32_t *dtype, void **dev_ptr) {
    QS_API_BEGIN
    if (!s) fail(QS_ERR_INVALID, "state is NULL");
    if (n_qubits) *n_qubits = s->d.n;
    if (dtype) *dtype = s->d.dtype;
    if (dev_ptr) *dev_ptr = s->d.psi;
    QS_API_END
}

int qs_apply_circuit(qs_state *s, const qs_gate *gates, size_t n_gates, const qs_options *opt) {
    QS_API_BEGIN
    if (!s) fail(QS_ERR_INVALID, "state is NULL");
    if (n_gates && !gates) fail(QS_ERR_INVALID, "gates is NULL");
    qs_options o{};
    if (opt) o = *opt;
    std::vector<Op> ops;
    ops.reserve(n_gates);
    for (size_t i = 0; i < n_gates; i++) {
        try {
            validate_gate(gates[i], s->d.n);
        } catch (const Error &e) {
            fail(e.code, "gate " + std::to_string(i) + ": " + e.msg);
        }
    }
    for (size_t i = 0; i < n_gates; i++) ops.push_back(lower_gate(gates[i]));
    execute(s, ops, o);
    QS_API_END
}

int qs_plan(int n_qubits, qs_dtype dt, const qs_gate *gates, size_t n_gates, const qs_options *opt,
            int32_t *pass_of_gate, uint64_t *pass_lmask, int64_t *n_passes) {
    QS_API_BEGIN
    if (n_qubits < 1 || n_qubits > QS_MAX_QUBITS) fail(QS_ERR_INVALID, "n_qubits out of range");
    if (dt != QS_C64 && dt != QS_C128) fail(QS_ERR_INVALID, "unknown dtype");
    if (n_gates && (!gates || !pass_of_gate || !pass_lmask)) fail(QS_ERR_INVALID, "NULL argument");
    if (!n_passes) fail(QS_ERR_INVALID, "NULL argument");
    qs_options o{};
    if (opt) o = *opt;
    std::vector<Op> ops;
    for (size_t i = 0; i < n_gates; i++) {
        try {
            validate_gate(gates[i], n_qubits);
        } catch (const Error &e) {
            fail(e.code, "gate " + std::to_string(i) + ": " + e.msg);
        }
        ops.push_back(lower_gate(gates[i]));
    }
    DeviceState d;
    d.n = n_qubits;
    d.dtype = dt;
    d.reg_phases = (o.flags & QS_OPT_NO_REG_PHASES) == 0;
    std::vector<Op> merged;
    std::vector<std::pair<size_t, size_t>> origin;
    const std::vector<Pass> plan = choose_plan(ops, n_qubits, plan_params(d, o), o, merged, origin);
    for (size_t p = 0; p < plan.size(); p++) {
        pass_lmask[p] = plan[p].stream ? 0 : plan[p].lmask;
        for (int i : plan[p].ops) {
            if (merged.empty()) {
                pass_of_gate[i] = (int32_t)p;
            } else {
                for (size_t g = origin[i].first; g < origin[i].second; g++) pass_of_gate[g] = (int32_t)p;
            }
        }
    }
    *n_passes = (int64_t)plan.size();
    QS_API_END
}

int qs_last_stats(const qs_state *s, qs_stats *out) {
    QS_API_BEGIN
    if (!s || !out) fail(QS_ERR_INVALID, "NULL argument");
    *out = s->stats;
    QS_API_END
}

int qs_set_amplitudes(qs_state *s, uint64_t off, uint64_t cnt, const void *host_src) {
    QS_API_BEGIN
    if (!s || (cnt && !host_src)) fail(QS_ERR_INVALID, "NULL argument");
    const uint64_t N = 1ull << s->d.n;
    if (off > N || cnt > N - off) fail(QS_ERR_INVALID, "amplitude range out of bounds");
    const size_t B = amp_bytes(s->d.dtype);
    copy_host(s->d, (char *)s->d.psi + off * B, host_src, cnt * B, true, 0);
    QS_CUDA(cudaStreamSynchronize(s->d.stream));
    QS_API_END
}

int qs_amplitudes(qs_state *s, uint64_t off, uint64_t cnt, void *host_dst) {
    QS_API_BEGIN
    if (!s || (cnt && !host_dst)) fail(QS_ERR_INVALID, "NULL argument");
    const uint64_t N = 1ull << s->d.n;
    if (off > N || cnt > N - off) fail(QS_ERR_INVALID, "amplitude range out of bounds");
    const size_t B = amp_bytes(s->d.dtype);
    sync_and_check(s->d);
    copy_host(s->d, host_dst, (const char *)s->d.psi + off * B, cnt * B, false, 0);
    QS_CUDA(cudaStreamSynchronize(s->d.stream));
    QS_API_END
}

int qs_set_amplitudes_async(qs_state *s, uint64_t off, uint64_t cnt, const void *host_src) {
    QS_API_BEGIN
    if (!s || (cnt && !host_src)) fail(QS_ERR_INVALID, "NULL argument");
    const uint64_t N = 1ull << s->d.n;
    if (off > N || cnt > N - off) fail(QS_ERR_INVALID, "amplitude range out of bounds");
    const size_t B = amp_bytes(s->d.dtype);
    copy_host(s->d, (char *)s->d.psi + off * B, host_src, cnt * B, true, kCopyEngines);
    QS_API_END
}

int qs_amplitudes_async(qs_state *s, uint64_t off, uint64_t cnt, void *host_dst) {
    QS_API_BEGIN
    if (!s || (cnt && !host_dst)) fail(QS_ERR_INVALID, "NULL argument");
    const uint64_t N = 1ull << s->d.n;
    if (off > N || cnt > N - off) fail(QS_ERR_INVALID, "amplitude range out of bounds");
    const size_t B = amp_bytes(s->d.dtype);
    copy_host(s->d, host_dst, (const char *)s->d.psi + off * B, cnt * B, false, kCopyEngines);
    QS_API_END
}

int qs_norm(qs_state *s, double *out) {
    QS_API_BEGIN
    if (!s || !out) fail(QS_ERR_INVALID, "NULL argument");
    reduce_expz(s->d, out, nullptr);
    QS_API_END
}

int qs_expectation_z(qs_state *s, double *out, double *norm_out) {
    QS_API_BEGIN
    if (!s || !out) fail(QS_ERR_INVALID, "NULL argument");
    double nrm = 0.0;
    reduce_expz(s->d, &nrm, out);
    if (norm_out) *norm_out = nrm;
    QS_API_END
}

int qs_top_amplitudes(qs_state *s, uint32_t k, uint64_t *idx, double *amp) {
    QS_API_BEGIN
    if (!s || (k && (!idx || !amp))) fail(QS_ERR_INVALID, "NULL argument");
    top_k(s->d, k, idx, amp);
    QS_API_END
}

int qs_renormalize(qs_state *s, double *old_norm) {
    QS_API_BEGIN
    if (!s) fail(QS_ERR_INVALID, "state is NULL");
    double nrm = 0.0;
    reduce_expz(s->d, &nrm, nullptr);
    if (!(nrm > 0.0)) fail(QS_ERR_INVALID, "state has zero norm");
    launch_scale(s->d, 1.0 / std::sqrt(nrm));
    QS_CUDA(cudaStreamSynchronize(s->d.stream));
    if (old_norm) *old_norm = nrm;
    QS_API_END
}

}  // extern "C"
