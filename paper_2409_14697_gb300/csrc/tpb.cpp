// Tensor Product Booster (QueenV2 Sec. III-A tier 1, the first stage of the all-in-one
// module; Sec. III-B notes it rests on the definition of the tensor product).  The paper
// names the stage and says it is inspired by merge sort, but does not publish it; this is
// our reading.
//
// A state known to be |0...0> is a product state.  Gates applied to it keep it a product
// of independent parts as long as no gate couples two parts: the qubits form components
// (union-find over each gate's operands) and the state of the prefix is the tensor product
// of one sub-state per component.  The booster takes the longest such prefix that keeps
// every component within kTpbMaxComponent qubits (a gate that would exceed it, or that
// touches a qubit of a gate left out, is left for the rest of the circuit and blocks its
// qubits; every gate taken shares no qubit with a gate left out before it, so it may move
// ahead of them).  Components are packed into at most kTpbMaxGroups groups of at most
// kTpbGroupQubits qubits (first fit, largest first).  Each group's sub-state is built by
// the ordinary executor on a small state of that many qubits (its gates relabelled onto
// qubits 0..k-1, from |0...0>); components within a group stay independent there, so the
// group's state is their tensor product.  One write pass then forms every amplitude as the
// product of one entry per group (k_tpb.cu): pairwise merging as in merge sort, the last
// merge written straight into the state.
#include <algorithm>

#include "plan.h"
#include "tpb.h"

namespace qs {

TpbPlan tpb_find(const std::vector<Op> &ops, int n, int max_component, int group_qubits) {
    TpbPlan tp;
    const uint64_t all = (1ull << n) - 1ull;
    int parent[64], size[64];
    for (int q = 0; q < n; q++) {
        parent[q] = q;
        size[q] = 1;
    }
    auto root = [&](int q) {
        while (parent[q] != q) q = parent[q] = parent[parent[q]];
        return q;
    };
    uint64_t blocked = 0;
    for (size_t i = 0; i < ops.size() && blocked != all; i++) {
        const Op &op = ops[i];
        const uint64_t qm = op.qmask();
        if (op.kind == K_PHASEFN || (qm & blocked)) {
            blocked |= qm;
            continue;
        }
        int roots[8], nr = 0, tot = 0;
        for (int j = 0; j < op.k; j++) {
            const int r = root(op.q[j]);
            bool seen = false;
            for (int t = 0; t < nr; t++) seen |= roots[t] == r;
            if (!seen) {
                roots[nr++] = r;
                tot += size[r];
            }
        }
        if (tot > max_component) {
            blocked |= qm;
            continue;
        }
        for (int t = 1; t < nr; t++) {
            parent[roots[t]] = roots[0];
            size[roots[0]] += size[roots[t]];
        }
        tp.taken.push_back((int)i);
    }
    if (tp.taken.empty()) return tp;
    // components (every qubit is in one; untouched qubits are singletons in |0>)
    std::vector<std::pair<int, uint64_t>> comps;  // (size, mask)
    {
        uint64_t cmask[64] = {0};
        for (int q = 0; q < n; q++) cmask[root(q)] |= 1ull << q;
        for (int q = 0; q < n; q++)
            if (cmask[q]) comps.push_back({__builtin_popcountll(cmask[q]), cmask[q]});
    }
    std::stable_sort(comps.begin(), comps.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::vector<uint64_t> groups;
    for (const auto &c : comps) {
        bool placed = false;
        for (uint64_t &g : groups)
            if (__builtin_popcountll(g) + c.first <= group_qubits) {
                g |= c.second;
                placed = true;
                break;
            }
        if (!placed) groups.push_back(c.second);
    }
    if ((int)groups.size() > kTpbMaxGroups) {
        tp.taken.clear();
        return tp;
    }
    tp.group_mask = groups;
    tp.group_ops.resize(groups.size());
    for (int i : tp.taken) {
        const uint64_t qm = ops[i].qmask();
        for (size_t g = 0; g < groups.size(); g++)
            if (qm & groups[g]) {
                tp.group_ops[g].push_back(i);
                break;
            }
    }
    return tp;
}

std::vector<Op> tpb_group_ops(const std::vector<Op> &ops, const TpbPlan &tp, int g, int n) {
    const uint64_t gm = tp.group_mask[g];
    int local[64] = {0};
    for (int q = 0, r = 0; q < n; q++)
        if ((gm >> q) & 1ull) local[q] = r++;
    std::vector<Op> gops;
    gops.reserve(tp.group_ops[g].size());
    for (int i : tp.group_ops[g]) {
        Op op = ops[i];
        for (int j = 0; j < op.k; j++) op.q[j] = local[op.q[j]];
        gops.push_back(std::move(op));
    }
    return gops;
}

std::vector<Op> tpb_rest(const std::vector<Op> &ops, const TpbPlan &tp) {
    std::vector<char> taken(ops.size(), 0);
    for (int i : tp.taken) taken[i] = 1;
    std::vector<Op> rest;
    rest.reserve(ops.size() - tp.taken.size());
    for (size_t i = 0; i < ops.size(); i++)
        if (!taken[i]) rest.push_back(ops[i]);
    return rest;
}

void tpb_execute(DeviceState &st, const std::vector<Op> &ops, const TpbPlan &tp, const qs_options &o,
                 qs_stats &stats) {
    const size_t B = st.dtype == QS_C128 ? 16 : 8;
    const int G = (int)tp.group_mask.size();
    size_t need = 0;
    for (uint64_t g : tp.group_mask) need += ((B << __builtin_popcountll(g)) + 255) & ~size_t(255);
    if (st.tpb_buf_bytes < need) {  // stream-ordered: no wait for other streams' work
        if (st.tpb_buf) {
            QS_CUDA(cudaFreeAsync(st.tpb_buf, st.stream));
            st.tpb_buf = nullptr;
            st.tpb_buf_bytes = 0;
        }
        QS_CUDA(cudaMallocAsync(&st.tpb_buf, need, st.stream));
        st.tpb_buf_bytes = need;
    }
    const void *tables[kTpbMaxGroups];
    size_t off = 0;
    qs_options so = o;
    so.mode = QS_MODE_AUTO;
    for (int g = 0; g < G; g++) {
        const uint64_t gm = tp.group_mask[g];
        const int k = __builtin_popcountll(gm);
        if (!st.tpb_sub[g]) st.tpb_sub[g] = new DeviceState();
        DeviceState &sub = *st.tpb_sub[g];
        sub.psi = (char *)st.tpb_buf + off;
        sub.n = k;
        sub.dtype = st.dtype;
        sub.stream = st.stream;
        sub.dev_err = st.dev_err;  // bounded waits report through the state's error word
        tables[g] = sub.psi;
        off += ((B << k) + 255) & ~size_t(255);
        const std::vector<Op> gops = tpb_group_ops(ops, tp, g, st.n);
        launch_set_zero_state(sub);
        qs_stats ss{};
        if (!gops.empty()) run_circuit(sub, gops, so, ss);
        stats.bytes += ss.bytes;
    }
    launch_tpb_product(st, tables, tp.group_mask.data(), G);
    stats.passes++;
    stats.bytes += (double)B * (double)(1ull << st.n);  // one write of the state
    stats.tpb_gates += (int64_t)tp.taken.size();
}

void tpb_reserve(DeviceState &d, size_t arena_bytes) {
    for (int g = 0; g < kTpbMaxGroups; g++) {
        if (!d.tpb_sub[g]) d.tpb_sub[g] = new DeviceState();
        DeviceState &sub = *d.tpb_sub[g];
        sub.stream = d.stream;
        sub.dtype = d.dtype;
        arena_reserve(sub, arena_bytes);
    }
}

void tpb_free(DeviceState &d) {
    for (int g = 0; g < kTpbMaxGroups; g++) {
        if (!d.tpb_sub[g]) continue;
        d.tpb_sub[g]->dev_err = nullptr;  // owned by the parent state
        d.tpb_sub[g]->stream = nullptr;
        free_device_state(*d.tpb_sub[g]);
        delete d.tpb_sub[g];
        d.tpb_sub[g] = nullptr;
    }
    if (d.tpb_buf) cudaFreeAsync(d.tpb_buf, d.stream);
    d.tpb_buf = nullptr;
    d.tpb_buf_bytes = 0;
}

}  // namespace qs
