// Tensor Product Booster (QueenV2 Sec. III-A tier 1): host side (tpb.cpp).
#pragma once

#include "qs_internal.h"

namespace qs {

// Widest component (qubits coupled by the prefix's gates) the booster builds.
constexpr int kTpbMaxComponent = 14;
// Widest group sub-state (2^17 amplitudes: 2 MiB complex128).
constexpr int kTpbGroupQubits = 17;
// Smallest state the booster is tried on (below it a pass costs less than planning twice).
constexpr int kTpbMinQubits = 20;

struct TpbPlan {
    std::vector<int> taken;                   // ops built as a tensor product, in order
    std::vector<uint64_t> group_mask;         // qubits of each group
    std::vector<std::vector<int>> group_ops;  // the taken ops of each group, in order
};

// The booster's prefix of ops on an n-qubit |0...0> state (empty `taken`: none): components
// of at most max_component qubits, packed into at most kTpbMaxGroups groups of at most
// group_qubits qubits.
TpbPlan tpb_find(const std::vector<Op> &ops, int n, int max_component = kTpbMaxComponent,
                 int group_qubits = kTpbGroupQubits);
// The taken ops of group g on the group's own qubits 0..k-1 (a global qubit becomes its
// rank among the group's qubits).
std::vector<Op> tpb_group_ops(const std::vector<Op> &ops, const TpbPlan &tp, int g, int n);
// The ops the booster does not take, in order.
std::vector<Op> tpb_rest(const std::vector<Op> &ops, const TpbPlan &tp);
// Builds the prefix's state into st (overwriting every amplitude) on st.stream.
void tpb_execute(DeviceState &st, const std::vector<Op> &ops, const TpbPlan &tp, const qs_options &o,
                 qs_stats &stats);

}  // namespace qs
