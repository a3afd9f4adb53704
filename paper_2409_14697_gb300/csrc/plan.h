// Chunk planner + in-cache executor (QueenV2 Sec. II-B "Qubit Reordering", "In-cache
// Operations"; Sec. III-A tiers 4-5; Sec. III-B).
#pragma once

#include "qs_internal.h"

namespace qs {

struct PlanParams {
    int m;       // local qubits per chunk pass
    int c;       // low qubits always local (contiguous runs of 2^c amplitudes)
    int fuse_k;  // fusion width inside a pass
    double sweep_flops;  // fusion cost gate (see fuse_ops)
    bool tc;             // complex64 blocks of 4..6 qubits run on the tensor cores
    bool force_chunk;    // QS_MODE_CHUNK: single-op passes also run as chunk passes
    bool hi_diag = false;  // two-qubit diagonals may join with one qubit outside the local set
};

struct Pass {
    bool stream = false;    // run the ops with the streaming kernel (one launch each)
    uint64_t lmask = 0;     // local qubits of a chunk pass
    std::vector<int> ops;   // indices into the op list, in order
};

PlanParams plan_params(const DeviceState &st, const qs_options &o);
// Greedy dependency-respecting partition of ops into passes.
std::vector<Pass> make_plan(const std::vector<Op> &ops, int n, const PlanParams &pp);
// The plan QS_MODE_AUTO / CHUNK runs: the greedy plan of ops, or, if it needs fewer passes,
// the plan of ops with runs of diagonal gates merged into phase functions (then `merged`
// receives those ops and `origin` the input range each stands for; otherwise both are
// left empty).
std::vector<Pass> choose_plan(const std::vector<Op> &ops, int n, const PlanParams &pp, const qs_options &o,
                              std::vector<Op> &merged, std::vector<std::pair<size_t, size_t>> &origin);
// The ops one chunk pass applies, in order: the pass's gates, then
//  1. complex128: its Hadamards but the last run unscaled (exact at the pass's end);
//  2. fusion into dense blocks where that does not add arithmetic (gates with a qubit
//     outside the tile stay apart);
//  3. complex128 FP64 passes of 256 tiles or more: U3 as a real rotation between phases
//     that join the diagonal runs (smaller states are latency-bound: extra ops cost more);
//  4. runs of diagonal gates (a QFT target's controlled phases, the phases of step 3) as
//     diagonal blocks of up to 8 tile qubits, with factors for qubits outside the tile
//     (complex64 register phases hold one- and two-qubit diagonals without a sweep).
// ops: the list the pass's indices refer to (choose_plan's merged list where it made one).
std::vector<Op> pass_program(const DeviceState &st, const PlanParams &pp, const Pass &p, const std::vector<Op> &ops);
// One chunk pass over lmask applying ops already fused (tensor cores if use_tc); the
// tensor-core blocks and their operations are added to tc_stats.
int launch_pass_ops(DeviceState &st, uint64_t lmask, const std::vector<Op> &fused, bool use_tc,
                    qs_stats *tc_stats = nullptr);
// Plans `ops` into passes and launches them on st.stream, filling stats.
void run_planned(DeviceState &st, const std::vector<Op> &ops, const qs_options &o, qs_stats &stats);

}  // namespace qs
