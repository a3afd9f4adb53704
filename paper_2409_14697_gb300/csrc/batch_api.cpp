// C interface of the batched persistent execution (include/qs.h, qs_batch_*).
#include "batch.h"
#include "capi_util.h"

struct qs_batch {
    qs::Batch b;
};

using namespace qs;

static void destroy_batch(qs_batch *p) {
    Batch &b = p->b;
    if (b.stream) cudaStreamSynchronize(b.stream);
    if (b.exec) cudaGraphExecDestroy(b.exec);
    cudaFree(b.d_states);
    cudaFree(b.d_passes);
    cudaFree(b.d_ops);
    cudaFree(b.d_mats);
    cudaFree(b.d_counter);
    cudaFree(b.d_done);
    cudaFree(b.d_err);
    cudaFree(b.d_abort);
    if (b.owns_stream && b.stream) cudaStreamDestroy(b.stream);
    delete p;
}

extern "C" {

int qs_batch_create(const qs_circuit *circuits, size_t count, qs_dtype dt, const qs_options *opt,
                    qs_batch **out) {
    QS_API_BEGIN
    if (!out || (count && !circuits)) fail(QS_ERR_INVALID, "NULL argument");
    if (dt != QS_C64 && dt != QS_C128) fail(QS_ERR_INVALID, "unknown dtype");
    if (count == 0) fail(QS_ERR_INVALID, "empty batch");
    *out = nullptr;
    qs_options o{};
    if (opt) o = *opt;
    std::vector<std::vector<Op>> ops(count);
    std::vector<int> nq(count);
    for (size_t c = 0; c < count; c++) {
        const int n = circuits[c].n_qubits;
        if (n < 1 || n > 30) fail(QS_ERR_INVALID, "batched circuit qubit count out of range");
        if (circuits[c].n_gates && !circuits[c].gates) fail(QS_ERR_INVALID, "gates is NULL");
        nq[c] = n;
        for (uint64_t g = 0; g < circuits[c].n_gates; g++) {
            try {
                validate_gate(circuits[c].gates[g], n);
            } catch (const Error &e) {
                fail(e.code, "circuit " + std::to_string(c) + " gate " + std::to_string(g) + ": " + e.msg);
            }
            ops[c].push_back(lower_gate(circuits[c].gates[g]));
        }
    }
    qs_batch *p = new qs_batch();
    p->b.dtype = dt;
    p->b.nq = nq;
    try {
        QS_CUDA(cudaStreamCreateWithFlags(&p->b.stream, cudaStreamNonBlocking));
        batch_build(p->b, ops, nq, o);
        batch_capture(p->b);
    } catch (...) {
        destroy_batch(p);
        throw;
    }
    *out = p;
    QS_API_END
}

int qs_batch_run(qs_batch *p) {
    QS_API_BEGIN
    if (!p) fail(QS_ERR_INVALID, "batch is NULL");
    QS_CUDA(cudaGraphLaunch(p->b.exec, p->b.stream));
    count_launch();
    QS_API_END
}

int qs_batch_synchronize(qs_batch *p) {
    QS_API_BEGIN
    if (!p) fail(QS_ERR_INVALID, "batch is NULL");
    QS_CUDA(cudaStreamSynchronize(p->b.stream));
    int e = 0;
    QS_CUDA(cudaMemcpy(&e, p->b.d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
        QS_CUDA(cudaMemset(p->b.d_err, 0, sizeof(int)));
        QS_CUDA(cudaMemset(p->b.d_abort, 0, sizeof(int)));
        fail(e, "a bounded wait in the batched kernel gave up");
    }
    QS_API_END
}

int qs_batch_set_stream(qs_batch *p, void *stream) {
    QS_API_BEGIN
    if (!p) fail(QS_ERR_INVALID, "batch is NULL");
    QS_CUDA(cudaStreamSynchronize(p->b.stream));
    if (p->b.owns_stream) QS_CUDA(cudaStreamDestroy(p->b.stream));
    p->b.stream = (cudaStream_t)stream;
    p->b.owns_stream = false;
    QS_API_END
}

int qs_batch_amplitudes(qs_batch *p, uint64_t i, uint64_t off, uint64_t cnt, void *host_dst) {
    QS_API_BEGIN
    if (!p || (cnt && !host_dst)) fail(QS_ERR_INVALID, "NULL argument");
    const Batch &b = p->b;
    if (i >= b.nq.size()) fail(QS_ERR_INVALID, "circuit index out of range");
    const uint64_t N = 1ull << b.nq[i];
    if (off > N || cnt > N - off) fail(QS_ERR_INVALID, "amplitude range out of bounds");
    const size_t B = b.dtype == QS_C128 ? 16 : 8;
    QS_CUDA(cudaStreamSynchronize(b.stream));
    QS_CUDA(cudaMemcpy(host_dst, (const char *)b.d_states + (b.state_off[i] + off) * B, cnt * B,
                       cudaMemcpyDeviceToHost));
    QS_API_END
}

int qs_batch_info(const qs_batch *p, qs_batch_stats *out) {
    QS_API_BEGIN
    if (!p || !out) fail(QS_ERR_INVALID, "NULL argument");
    const Batch &b = p->b;
    out->circuits = (int64_t)b.nq.size();
    out->passes = (int64_t)b.passes.size();
    out->work_items = (int64_t)b.total_items;
    out->grid = b.grid;
    out->state_bytes = b.state_elems * (b.dtype == QS_C128 ? 16 : 8);
    QS_API_END
}

int qs_batch_destroy(qs_batch *p) {
    QS_API_BEGIN
    if (!p) fail(QS_ERR_INVALID, "batch is NULL");
    destroy_batch(p);
    QS_API_END
}

}  // extern "C"
