// Merged diagonal runs ("infinite" diagonal gate fusion, QueenV2 Sec. III-A tier 2): a run
// of consecutive diagonal gates, on any qubits, becomes one phase function applied in a
// single pass over the state.
#pragma once

#include <memory>

#include "qs_internal.h"

namespace qs {

// Every diagonal gate on at most two qubits is, exactly,
//     d(x) = C * beta_a^(x_a) * beta_b^(x_b) * delta^(x_a x_b)
// (C = d(00), beta_a = d(10)/d(00), beta_b = d(01)/d(00), delta = d(11) d(00) / (d(10) d(01))).
// The product over a run collects C, one beta per qubit and one delta per qubit pair; equal
// betas and equal deltas are grouped, and each group contributes value^count(x):
//   PF_WEIGHT: count = popcount(x & mask)           (a group of equal betas; when the
//              group carries a clique, also delta_c^(count (count - 1) / 2): every pair of
//              the mask with the same delta, e.g. fully connected QAOA)
//   PF_PAIRS:  count = #pairs (a, b) with x_a = x_b = 1   (a group of equal deltas)
// F(x) = table[sum_g count_g(x) * stride_g]; the table (at most kPfMaxTable entries) holds
// C times the product of every group's factor, so one multiply per amplitude applies it.
enum PfKind : int32_t { PF_WEIGHT = 0, PF_PAIRS = 1 };
constexpr int kPfMaxGroups = 6;
constexpr int kPfMaxTable = 4096;

struct PfGroup {
    PfKind kind;
    uint64_t mask = 0;                       // PF_WEIGHT
    std::vector<std::pair<int, int>> pairs;  // PF_PAIRS
    cd value = 1.0;                          // beta (weight) or delta (pairs)
    cd clique = 1.0;                         // PF_WEIGHT: delta of every pair in the mask
    int max_count = 0;
    int stride = 1;
};

struct PhaseFn {
    uint64_t qmask = 0;
    std::vector<PfGroup> groups;
    std::vector<cd> table;
};

// True if op is a diagonal on at most two qubits (the forms a phase function absorbs).
bool pf_absorbs(const Op &op);
// Builds the phase function of ops[begin, end) (all pf_absorbs); null if its table would
// exceed kPfMaxTable entries or kPfMaxGroups groups.
std::shared_ptr<const PhaseFn> build_phasefn(const std::vector<Op> &ops, size_t begin, size_t end);
// Replaces every run of at least min_run consecutive absorbable diagonals by one K_PHASEFN
// op (runs whose table is too large stay as they are).
// origin (optional) receives, per output op, the range [begin, end) of input ops it stands for.
std::vector<Op> merge_diagonal_runs(const std::vector<Op> &ops, int min_run,
                                    std::vector<std::pair<size_t, size_t>> *origin = nullptr);
// The phase-function pass handles states of at least 9 qubits (units of 2^9 amplitudes).
bool phasefn_supported(int n);

}  // namespace qs
