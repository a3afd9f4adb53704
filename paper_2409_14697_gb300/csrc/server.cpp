// C6: serving runtime with continuous batching (include/qs.h, qs_server_* / qs_submit /
// qs_poll).  The paper has no serving layer; this is the request loop around the hot path.
//
// Requests enter a FIFO queue.  A worker thread admits the queue head as soon as a slot
// is free and the bytes of the admitted states (2^n x bytes per amplitude) stay within
// the HBM budget; requests that arrive while others run are admitted as slots and memory
// free up.  Each slot owns a CUDA stream, so admitted requests overlap on the device.
// A request's work is queued on its slot's stream: stream-ordered state allocation
// (cudaMallocAsync), the initial state (|0...0> or the caller's amplitudes), the planned
// circuit, the <Z_q> reduction, top-K, and copies of the results into pinned host memory,
// then an event that the worker polls to timestamp completion.  The worker then retires
// the slot (stream-ordered free) and publishes the result.  All kernels are deterministic (no
// floating-point atomics, fixed reduction order, the plan depends only on the circuit),
// so a result is bitwise the same alone and in any mix.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "capi_util.h"
#include "qs_internal.h"

namespace qs {

struct Server;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    int n;
    int dtype;
    std::vector<Op> ops;
    std::vector<char> init;  // host amplitudes copied at submission (empty: none)
    const void *init_borrowed = nullptr;  // caller's amplitudes (QS_REQ_BORROW_INIT)
    uint32_t top_k;
    qs_options opt;
    Clock::time_point t_submit;
    size_t bytes;
};

struct Result {
    int status = QS_NOT_READY;
    std::string error;
    std::vector<double> expz;
    double norm = 0.0;
    std::vector<uint64_t> top_idx;
    std::vector<double> top_amp;
    double latency_s = 0.0;
    double queue_s = 0.0;
};

struct Slot {
    Server *srv = nullptr;
    DeviceState d;
    bool busy = false;
    uint64_t ticket = 0;
    size_t bytes = 0;
    uint32_t top_k = 0;
    int n = 0;
    Clock::time_point t_submit, t_start;
    // device result buffers (sized for the largest request seen) and pinned host mirrors
    double *d_out = nullptr;
    uint64_t *d_idx = nullptr;
    double *d_amp = nullptr;
    double *h_out = nullptr;
    uint64_t *h_idx = nullptr;
    double *h_amp = nullptr;
    int cap_n = 0;
    uint32_t cap_k = 0;
    void *h_init = nullptr;  // pinned staging of the initial amplitudes
    size_t h_init_cap = 0;
    int *h_err = nullptr;    // pinned copy of the slot's device error word
    cudaEvent_t ev_done = nullptr;  // recorded after the request's last operation
    void *own_psi = nullptr;        // small-lane slots: a state buffer of their own
    size_t own_psi_bytes = 0;
    Clock::time_point t_done;
};

}  // namespace

struct Server {
    qs_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Result> results;
    std::unordered_set<uint64_t> pending;  // submitted, result not yet delivered
    std::vector<Slot *> slots;
    size_t bytes_in_use = 0, peak_bytes = 0;
    uint64_t next_ticket = 1, submitted = 0, completed = 0, failed = 0;
    bool stop = false;
    std::thread worker;
    cudaMemPool_t pool = nullptr;

    void run();
    void start_request(Slot &s, Request &r);
    void finish_slot(Slot &s);
};

namespace {

size_t amp_bytes_of(int dtype) { return dtype == QS_C128 ? 16 : 8; }

}  // namespace

namespace {

// Result buffers of a slot for any request (QS_MAX_QUBITS + 1 values, 4096 amplitudes), so
// they never grow: growing frees memory, and cudaFree / cudaFreeHost wait for the whole
// device, which would stall the worker behind every request in flight.
void presize_results(Slot &s) {
    s.cap_n = QS_MAX_QUBITS;
    s.cap_k = 4096;
    QS_CUDA(cudaMalloc(&s.d_out, sizeof(double) * (s.cap_n + 1)));
    QS_CUDA(cudaMalloc(&s.d_idx, sizeof(uint64_t) * s.cap_k));
    QS_CUDA(cudaMalloc(&s.d_amp, sizeof(double) * 2 * s.cap_k));
    QS_CUDA(cudaMallocHost(&s.h_out, sizeof(double) * (s.cap_n + 1)));
    QS_CUDA(cudaMallocHost(&s.h_idx, sizeof(uint64_t) * s.cap_k));
    QS_CUDA(cudaMallocHost(&s.h_amp, sizeof(double) * 2 * s.cap_k));
}

// A small-lane slot: also scratch for requests of up to n qubits and top-k amplitudes, and
// parameter arenas of 1 MiB each, so small requests never grow (or free) anything.
void presize_slot(Slot &s, int n, uint32_t k) {
    DeviceState &d = s.d;
    d.n = n;
    const uint32_t kk = (uint32_t)std::min<uint64_t>(std::max<uint32_t>(k, 1), 1ull << n);
    ensure_scratch(d, std::max(scratch_expz_bytes(n), scratch_topk_bytes(n, kk)));
    presize_results(s);
    arena_reserve(d, (size_t)1 << 20);
}

}  // namespace

constexpr int kYieldIters = 16;

void Server::start_request(Slot &s, Request &r) {
    DeviceState &d = s.d;
    d.n = r.n;
    d.dtype = r.dtype;
    const size_t state_bytes = r.bytes;
    const bool own = s.own_psi && state_bytes <= s.own_psi_bytes;
    if (own) d.psi = s.own_psi;
    else QS_CUDA(cudaMallocFromPoolAsync(&d.psi, state_bytes, pool, d.stream));
    d.known_zero = false;
    if (r.init_borrowed) {
        QS_CUDA(cudaMemcpyAsync(d.psi, r.init_borrowed, state_bytes, cudaMemcpyHostToDevice, d.stream));
    } else if (r.init.empty()) {
        launch_set_zero_state(d);
    } else {
        if (s.h_init_cap < state_bytes) {
            if (s.h_init) {
                QS_CUDA(cudaStreamSynchronize(d.stream));
                QS_CUDA(cudaFreeHost(s.h_init));
            }
            QS_CUDA(cudaMallocHost(&s.h_init, state_bytes));
            s.h_init_cap = state_bytes;
        }
        std::memcpy(s.h_init, r.init.data(), state_bytes);
        QS_CUDA(cudaMemcpyAsync(d.psi, s.h_init, state_bytes, cudaMemcpyHostToDevice, d.stream));
    }
    qs_stats st{};
    {
        // with a small-request lane, a larger request's gate kernels run as grids whose blocks
        // loop over at most kYieldIters work blocks (tiles, or groups of amplitudes for 256
        // threads), about 0.1-1 ms each, so that a small request's kernels on their
        // high-priority streams start within a block's time instead of a launch's
        const bool yield = cfg.small_slots > 0 && r.n > cfg.small_max_qubits;
        LaunchYield ly(yield ? kYieldIters : 0);
        run_circuit(d, r.ops, r.opt, st);
    }
    // results
    if (s.cap_n < r.n || s.cap_k < r.top_k) {
        QS_CUDA(cudaStreamSynchronize(d.stream));
        cudaFree(s.d_out); cudaFree(s.d_idx); cudaFree(s.d_amp);
        cudaFreeHost(s.h_out); cudaFreeHost(s.h_idx); cudaFreeHost(s.h_amp);
        s.cap_n = std::max(s.cap_n, r.n);
        s.cap_k = std::max<uint32_t>(s.cap_k, std::max<uint32_t>(r.top_k, 1));
        QS_CUDA(cudaMalloc(&s.d_out, sizeof(double) * (s.cap_n + 1)));
        QS_CUDA(cudaMalloc(&s.d_idx, sizeof(uint64_t) * s.cap_k));
        QS_CUDA(cudaMalloc(&s.d_amp, sizeof(double) * 2 * s.cap_k));
        QS_CUDA(cudaMallocHost(&s.h_out, sizeof(double) * (s.cap_n + 1)));
        QS_CUDA(cudaMallocHost(&s.h_idx, sizeof(uint64_t) * s.cap_k));
        QS_CUDA(cudaMallocHost(&s.h_amp, sizeof(double) * 2 * s.cap_k));
    }
    ensure_scratch(d, std::max(scratch_expz_bytes(r.n), scratch_topk_bytes(r.n, std::max<uint32_t>(r.top_k, 1))));
    reduce_expz_async(d, s.d_out);
    if (r.top_k) top_k_async(d, r.top_k, s.d_idx, s.d_amp);
    QS_CUDA(cudaMemcpyAsync(s.h_out, s.d_out, sizeof(double) * (r.n + 1), cudaMemcpyDeviceToHost, d.stream));
    if (r.top_k) {
        QS_CUDA(cudaMemcpyAsync(s.h_idx, s.d_idx, sizeof(uint64_t) * r.top_k, cudaMemcpyDeviceToHost, d.stream));
        QS_CUDA(cudaMemcpyAsync(s.h_amp, s.d_amp, sizeof(double) * 2 * r.top_k, cudaMemcpyDeviceToHost, d.stream));
    }
    QS_CUDA(cudaMemcpyAsync(s.h_err, d.dev_err, sizeof(int), cudaMemcpyDeviceToHost, d.stream));
    if (!own) QS_CUDA(cudaFreeAsync(d.psi, d.stream));
    d.psi = nullptr;
    // completion is polled with the event (host functions of independent streams may run
    // one after the other in launch order, which would finish a small request only after
    // every large one launched before it)
    QS_CUDA(cudaEventRecord(s.ev_done, d.stream));
}

void Server::finish_slot(Slot &s) {
    Result res;
    res.status = QS_OK;
    res.norm = s.h_out[0];
    res.expz.assign(s.h_out + 1, s.h_out + 1 + s.n);
    res.top_idx.assign(s.h_idx, s.h_idx + s.top_k);
    res.top_amp.assign(s.h_amp, s.h_amp + 2 * s.top_k);
    // the device error word (bounded waits) of this slot
    if (*s.h_err) {
        res.status = *s.h_err;
        res.error = "a bounded device-side wait gave up";
        *s.h_err = 0;
        cudaMemsetAsync(s.d.dev_err, 0, sizeof(int), s.d.stream);
    }
    res.latency_s = std::chrono::duration<double>(s.t_done - s.t_submit).count();
    res.queue_s = std::chrono::duration<double>(s.t_start - s.t_submit).count();
    std::lock_guard<std::mutex> lk(mu);
    results[s.ticket] = std::move(res);
    bytes_in_use -= s.bytes;
    completed++;
    s.busy = false;
    cv.notify_all();
}

void Server::run() {
    cudaSetDevice(device);
    for (;;) {
        // 1. retire finished slots
        for (Slot *s : slots) {
            if (!s->busy) continue;
            const cudaError_t q = cudaEventQuery(s->ev_done);
            if (q == cudaErrorNotReady) {
                cudaGetLastError();  // not an error: clear it so later launch checks do not see it
                continue;
            }
            s->t_done = Clock::now();
            if (q != cudaSuccess && *s->h_err == 0) *s->h_err = QS_ERR_CUDA;
            finish_slot(*s);
        }
        // 2. admit: large requests in submission order (the first that cannot start holds
        // back the later large ones); small requests whenever a slot and the budget allow,
        // small-lane slots first
        std::unique_lock<std::mutex> lk(mu);
        // starts one queued request (mu held; released while the request is queued on its
        // slot's stream); false if none can start now
        auto admit_one = [&]() -> bool {
            bool large_blocked = false;
            for (auto it = queue.begin(); it != queue.end(); ++it) {
                const bool small = it->n <= cfg.small_max_qubits;
                if ((!small && large_blocked) || bytes_in_use + it->bytes > cfg.hbm_budget_bytes) {
                    large_blocked |= !small;
                    continue;
                }
                Slot *free_slot = nullptr;
                const int n_regular = cfg.max_slots;
                if (small)
                    for (size_t i = n_regular; i < slots.size() && !free_slot; i++)
                        if (!slots[i]->busy) free_slot = slots[i];
                for (int i = 0; i < n_regular && !free_slot; i++)
                    if (!slots[i]->busy) free_slot = slots[i];
                if (!free_slot) {
                    large_blocked |= !small;
                    continue;
                }
                Request req = std::move(*it);
                queue.erase(it);  // iterators are not used again: the lock is released below
                free_slot->busy = true;
                free_slot->ticket = req.ticket;
                free_slot->bytes = req.bytes;
                free_slot->top_k = req.top_k;
                free_slot->n = req.n;
                free_slot->t_submit = req.t_submit;
                free_slot->t_start = Clock::now();
                bytes_in_use += req.bytes;
                peak_bytes = std::max(peak_bytes, bytes_in_use);
                lk.unlock();
                try {
                    start_request(*free_slot, req);
                } catch (const Error &e) {
                    lk.lock();
                    Result res;
                    res.status = e.code;
                    res.error = e.msg;
                    results[req.ticket] = std::move(res);
                    bytes_in_use -= req.bytes;
                    failed++;
                    completed++;
                    free_slot->busy = false;
                    cv.notify_all();
                    lk.unlock();
                }
                lk.lock();
                return true;
            }
            return false;
        };
        bool admitted = false;
        while (admit_one()) admitted = true;
        if (stop && queue.empty()) {
            bool any = false;
            for (Slot *s : slots) any |= s->busy;
            if (!any) return;
        }
        bool any_busy = false;
        for (Slot *s : slots) any_busy |= s->busy;
        if (!admitted) {
            // wait for a submission (it notifies), or poll the busy slots' events again
            cv.wait_for(lk, any_busy ? std::chrono::microseconds(200) : std::chrono::microseconds(20000));
        }
    }
}

}  // namespace qs

struct qs_server {
    qs::Server s;
};

using namespace qs;

extern "C" {

int qs_server_create(const qs_server_config *cfg, qs_server **out) {
    QS_API_BEGIN
    if (!cfg || !out) fail(QS_ERR_INVALID, "NULL argument");
    if (cfg->max_slots < 1 || cfg->max_slots > 256) fail(QS_ERR_INVALID, "max_slots must be 1..256");
    if (cfg->small_slots < 0 || cfg->small_slots > 256) fail(QS_ERR_INVALID, "small_slots must be 0..256");
    if (cfg->hbm_budget_bytes == 0) fail(QS_ERR_INVALID, "zero HBM budget");
    *out = nullptr;
    qs_server *p = new qs_server();
    Server &S = p->s;
    S.cfg = *cfg;
    try {
        QS_CUDA(cudaGetDevice(&S.device));
        // a pool of the server's own for the request states: freed state memory stays in it for
        // reuse, but an allocation never reuses memory whose free is still pending on another
        // slot's stream (that would make the new request wait for the old one's work)
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = S.device;
        QS_CUDA(cudaMemPoolCreate(&S.pool, &props));
        uint64_t thr = UINT64_MAX;
        QS_CUDA(cudaMemPoolSetAttribute(S.pool, cudaMemPoolAttrReleaseThreshold, &thr));
        int no_wait = 0;
        QS_CUDA(cudaMemPoolSetAttribute(S.pool, cudaMemPoolReuseAllowInternalDependencies, &no_wait));
        // small-lane slots get the device's highest stream priority: when the persistent
        // kernels of a large request end, the CTA scheduler starts a small request's pending
        // kernels first instead of the large request's next pass
        int prio_low = 0, prio_high = 0;
        QS_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
        for (int i = 0; i < cfg->max_slots + cfg->small_slots; i++) {
            Slot *s = new Slot();
            S.slots.push_back(s);
            QS_CUDA(cudaStreamCreateWithPriority(&s->d.stream, cudaStreamNonBlocking,
                                                 i < cfg->max_slots ? prio_low : prio_high));
            s->srv = &S;
            QS_CUDA(cudaMalloc(&s->d.dev_err, sizeof(int)));
            QS_CUDA(cudaMemset(s->d.dev_err, 0, sizeof(int)));
            QS_CUDA(cudaMallocHost(&s->h_err, sizeof(int)));
            *s->h_err = 0;
            QS_CUDA(cudaEventCreateWithFlags(&s->ev_done, cudaEventDisableTiming));
            // small slots: scratch and arenas for their largest request; every slot: result
            // buffers for any request (at most QS_MAX_QUBITS values and 4096 amplitudes),
            // parameter arenas and the booster's sub-states.  Page-locked and plain device
            // allocations make the device finish other streams' work first, so a request
            // must not need one while others run.
            if (i >= cfg->max_slots && cfg->small_max_qubits > 0) {
                const int ns = std::min(cfg->small_max_qubits, 30);
                presize_slot(*s, ns, 4096);
                s->own_psi_bytes = (size_t)16 << ns;  // the largest small state, either dtype
                QS_CUDA(cudaMalloc(&s->own_psi, s->own_psi_bytes));
            } else {
                presize_results(*s);
                arena_reserve(s->d, (size_t)4 << 20);
                tpb_reserve(s->d, (size_t)256 << 10);
            }
        }
        // grow the pool to the budget now (at most 90 % of the free memory): a pool that grows
        // while requests run allocates device memory, and that makes the device finish the
        // other slots' work first
        {
            size_t free_b = 0, total_b = 0;
            QS_CUDA(cudaMemGetInfo(&free_b, &total_b));
            const size_t reserve = std::min<size_t>(cfg->hbm_budget_bytes, free_b / 10 * 9);
            void *p = nullptr;
            cudaStream_t s0 = S.slots[0]->d.stream;
            QS_CUDA(cudaMallocFromPoolAsync(&p, reserve, S.pool, s0));
            QS_CUDA(cudaFreeAsync(p, s0));
            QS_CUDA(cudaStreamSynchronize(s0));
        }
        S.worker = std::thread([&S]() { S.run(); });
    } catch (...) {
        for (Slot *s : S.slots) {
            free_device_state(s->d);
            if (s->own_psi) cudaFree(s->own_psi);
            if (s->d.stream) cudaStreamDestroy(s->d.stream);
            delete s;
        }
        if (S.pool) cudaMemPoolDestroy(S.pool);
        delete p;
        throw;
    }
    *out = p;
    QS_API_END
}

int qs_submit(qs_server *p, const qs_request *req, uint64_t *ticket) {
    QS_API_BEGIN
    if (!p || !req || !ticket) fail(QS_ERR_INVALID, "NULL argument");
    Server &S = p->s;
    const int n = req->n_qubits;
    if (n < 1 || n > QS_MAX_QUBITS) fail(QS_ERR_INVALID, "n_qubits out of range");
    if (req->dtype != QS_C64 && req->dtype != QS_C128) fail(QS_ERR_INVALID, "unknown dtype");
    if (req->n_gates && !req->gates) fail(QS_ERR_INVALID, "gates is NULL");
    if ((uint64_t)req->top_k > (1ull << n) || req->top_k > 4096) fail(QS_ERR_INVALID, "top_k exceeds min(2^n, 4096)");
    Request r;
    r.n = n;
    r.dtype = req->dtype;
    r.bytes = amp_bytes_of(req->dtype) << n;
    if (r.bytes > S.cfg.hbm_budget_bytes)
        fail(QS_ERR_NOMEM, "request needs " + std::to_string(r.bytes) + " bytes, more than the whole HBM budget");
    for (uint64_t g = 0; g < req->n_gates; g++) {
        try {
            validate_gate(req->gates[g], n);
        } catch (const Error &e) {
            fail(e.code, "gate " + std::to_string(g) + ": " + e.msg);
        }
        r.ops.push_back(lower_gate(req->gates[g]));
    }
    if (req->flags & ~(uint32_t)QS_REQ_BORROW_INIT) fail(QS_ERR_INVALID, "unknown request flags");
    if (req->init_amplitudes && (req->flags & QS_REQ_BORROW_INIT)) {
        r.init_borrowed = req->init_amplitudes;
    } else if (req->init_amplitudes) {
        r.init.resize(r.bytes);
        std::memcpy(r.init.data(), req->init_amplitudes, r.bytes);
    }
    r.top_k = req->top_k;
    r.opt = qs_options{};
    r.opt.mode = req->mode;
    r.opt.precision = req->precision;
    r.t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(S.mu);
    if (S.stop) fail(QS_ERR_BUSY, "server is shutting down");
    r.ticket = S.next_ticket++;
    *ticket = r.ticket;
    S.pending.insert(r.ticket);
    S.submitted++;
    S.queue.push_back(std::move(r));
    S.cv.notify_all();
    QS_API_END
}

int qs_poll(qs_server *p, uint64_t ticket, double *expz, double *norm, uint64_t *top_idx, double *top_amp,
            double *latency_s) {
    int rc = QS_OK;
    QS_API_BEGIN
    if (!p) fail(QS_ERR_INVALID, "server is NULL");
    Server &S = p->s;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.results.find(ticket);
    if (it == S.results.end()) {
        if (!S.pending.count(ticket)) fail(QS_ERR_INVALID, "unknown or already delivered ticket");
        rc = QS_NOT_READY;
    } else {
        Result &r = it->second;
        S.pending.erase(ticket);
        if (r.status < 0) {
            const int code = r.status;
            const std::string msg = r.error;
            S.results.erase(it);
            fail(code, msg);
        }
        if (expz) std::copy(r.expz.begin(), r.expz.end(), expz);
        if (norm) *norm = r.norm;
        if (top_idx) std::copy(r.top_idx.begin(), r.top_idx.end(), top_idx);
        if (top_amp) std::copy(r.top_amp.begin(), r.top_amp.end(), top_amp);
        if (latency_s) *latency_s = r.latency_s;
        S.results.erase(it);
    }
    QS_API_END_RC(rc)
}

int qs_server_stats(qs_server *p, qs_server_stats_t *out) {
    QS_API_BEGIN
    if (!p || !out) fail(QS_ERR_INVALID, "NULL argument");
    Server &S = p->s;
    std::lock_guard<std::mutex> lk(S.mu);
    out->submitted = S.submitted;
    out->completed = S.completed;
    out->failed = S.failed;
    out->queued = S.queue.size();
    out->bytes_in_use = S.bytes_in_use;
    out->peak_bytes = S.peak_bytes;
    int64_t busy = 0;
    for (Slot *s : S.slots) busy += s->busy;
    out->in_flight = busy;
    QS_API_END
}

int qs_server_drain(qs_server *p, double timeout_s) {
    QS_API_BEGIN
    if (!p) fail(QS_ERR_INVALID, "server is NULL");
    Server &S = p->s;
    std::unique_lock<std::mutex> lk(S.mu);
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (S.completed < S.submitted) {
        if (S.cv.wait_until(lk, until) == std::cv_status::timeout && S.completed < S.submitted)
            fail(QS_ERR_TIMEOUT, "requests still in flight after the timeout");
    }
    QS_API_END
}

int qs_server_destroy(qs_server *p) {
    QS_API_BEGIN
    if (!p) fail(QS_ERR_INVALID, "server is NULL");
    Server &S = p->s;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        bool busy = !S.queue.empty();
        for (Slot *s : S.slots) busy |= s->busy;
        if (busy) fail(QS_ERR_BUSY, "requests still queued or in flight (drain first)");
        S.stop = true;
        S.cv.notify_all();
    }
    if (S.worker.joinable()) S.worker.join();
    for (Slot *s : S.slots) {
        if (s->d.stream) cudaStreamSynchronize(s->d.stream);
        free_device_state(s->d);
        cudaFree(s->d_out); cudaFree(s->d_idx); cudaFree(s->d_amp);
        cudaFreeHost(s->h_out); cudaFreeHost(s->h_idx); cudaFreeHost(s->h_amp);
        if (s->h_init) cudaFreeHost(s->h_init);
        if (s->h_err) cudaFreeHost(s->h_err);
        if (s->ev_done) cudaEventDestroy(s->ev_done);
        if (s->own_psi) cudaFree(s->own_psi);
        if (s->d.stream) cudaStreamDestroy(s->d.stream);
        delete s;
    }
    if (S.pool) {
        cudaDeviceSynchronize();  // the pool's last frees are stream-ordered
        cudaMemPoolDestroy(S.pool);
    }
    delete p;
    QS_API_END
}

}  // extern "C"
