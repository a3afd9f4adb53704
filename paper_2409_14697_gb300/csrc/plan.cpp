// Chunk planner and executor (QueenV2 Sec. II-B "Qubit Reordering" and "In-cache
// Operations"; Sec. III-A tiers 4-5 "In-Rank" gate blocks and general fusion).
//
// The planner partitions the op sequence into passes.  A pass owns a set L of m local
// qubits that always contains the low c qubits (so every tile is made of contiguous
// runs of 2^c amplitudes in HBM) plus high qubits taken by the ops it accepts.  An op
// joins the pass if none of its qubits is blocked by an earlier op left for a later pass
// and its qubits fit in L; otherwise its qubits become blocked (ops on disjoint qubits
// commute, so later ops on other qubits may still join).  Several candidate passes are
// built: unrestricted (high qubits claimed in circuit order) and restricted to each
// window of m - c consecutive high qubits; the one that executes the most ops is kept.
// Qubit reordering is logical: the pass's local qubits are mapped to tile positions by
// a position table (the bidirectional qubit table of Sec. III-A) and the state is never
// permuted in memory.  Inside a pass, consecutive ops are fused into dense blocks of at
// most fuse_k qubits (FP64 host products) before the kernel applies them in shared
// memory.  A pass holding a single op runs on the streaming kernel instead, which
// touches only the amplitudes that op changes.
#include <algorithm>
#include <cmath>

#include "chunk.h"
#include "kgeom.h"
#include "phasefn.h"
#include "plan.h"
#include "tpb.h"

namespace qs {

namespace {

// Shortest run of consecutive diagonal gates worth merging into a phase function.
constexpr int kMinMergedRun = 4;
// Widest diagonal block merged inside a tile pass (its table: 2^8 entries, 512 reals).
constexpr int kTileDiagQubits = 8;

// Ops the shared-memory path applies: dense blocks up to 4 qubits (512 matrix reals)
// and diagonals up to 8 qubits.
bool chunkable(const Op &op, const PlanParams &pp) {
    if (op.kind == K_PHASEFN) return false;  // one streaming pass over the whole state
    if (op.kind == K_DENSE) return op.k <= 4 || (pp.tc && tc_available(pp.m, op.k));
    if (op.kind == K_DIAG) return op.k <= 8;
    return true;
}

}  // namespace

// Launches one chunk pass over lmask applying `fused` (tensor cores where allowed);
// returns the number of tile sweeps and adds the tensor-core blocks and their operations
// to *tc_stats.
int launch_pass_ops(DeviceState &st, uint64_t lmask, const std::vector<Op> &fused, bool use_tc,
                    qs_stats *tc_stats) {
    const int n = st.n;
    int pos[64] = {0};
    int r = 0;
    for (int b = 0; b < n; b++)
        if ((lmask >> b) & 1ull) pos[b] = r++;
    const int m = r;
    std::vector<KOp> kops;
    std::vector<double> mats;
    if (!use_tc && st.dtype == QS_C64 && st.reg_phases && rphase_applicable(m, kTileThreadBits)) {
        const std::vector<KOp> kp = build_register_phases(fused, pos, m, kTileThreadBits, mats);
        launch_chunk_pass(st, lmask, kp, mats);
        return (int)kp.size();
    }
    std::vector<float> bmats;
    uint32_t b_floats = 0;
    bool any_tc = false;
    for (const Op &op : fused)
        if ((op.qmask() & ~lmask) != 0)  // non-local qubits only as terms of diagonal blocks
            fail(QS_ERR_INVALID, "internal: op with a qubit outside the pass's local set");
    for (const Op &op : fused) {
        if (use_tc && op.kind == K_DENSE && tc_available(m, op.k)) {
            KOp k{};
            k.fkind = F_TC;
            k.k = op.k;
            for (int j = 0; j < op.k; j++) k.pos[j] = pos[op.q[j]];
            int off = 0, cnt = 0;
            build_tc_operand(op.m, op.k, bmats, off, cnt);
            k.mat = off;
            k.nmat = cnt;
            b_floats = std::max<uint32_t>(b_floats, (uint32_t)(cnt / 2));
            kops.push_back(k);
            any_tc = true;
            if (tc_stats) {
                // 2^(n-k) groups x 2^(k+1) x 2^(k+1) real multiply-adds, three TF32 products
                tc_stats->tc_blocks++;
                tc_stats->tc_flops += 6.0 * std::ldexp(1.0, st.n + op.k + 2);
            }
        } else {
            kops.push_back(make_tile_kop(op, pos, mats));
        }
    }
    if (!any_tc && st.dtype == QS_C128 && st.prec == QS_PREC_FP64) kops = join_h_cdiag(kops, mats);
    if (any_tc) launch_chunk_pass_tc(st, lmask, kops, mats, bmats, b_floats);
    else launch_chunk_pass(st, lmask, kops, mats);
    return (int)kops.size();
}

PlanParams plan_params(const DeviceState &st, const qs_options &o) {
    PlanParams p;
    const bool c128 = st.dtype == QS_C128;
    p.m = o.chunk_m > 0 ? o.chunk_m : (c128 ? 12 : 13);
    // complex128 passes are bound by the FP64 pipe of the SMs that hold tiles: a small
    // state (18 qubits and less) gets about 64 tiles, so that many SMs share its work (the
    // extra passes are cheap: such a state stays in L2)
    if (c128 && o.chunk_m <= 0) p.m = std::max(7, std::min(p.m, st.n - 6));
    p.c = c128 ? 4 : 5;                  // runs of 256 bytes
    p.m = std::min(p.m, st.n);
    p.c = std::min(p.c, p.m);
    // the shared-memory dense path applies blocks of at most 4 qubits; complex64 register
    // phases apply gates unfused (a fused block costs more flops than its members there)
    const bool phases = !c128 && st.reg_phases && rphase_applicable(p.m, kTileThreadBits);
    p.fuse_k = std::min(o.fuse_k > 0 ? o.fuse_k : (phases ? 1 : 2), 4);
    // FP64 is 1/72 of FP32 on GB300: for complex128 FP64 a fused block must not add flops;
    // double-float and complex64 arithmetic run on the FP32 pipe and are cheap next to a
    // shared-memory sweep of the tile (double-float applies every one-qubit matrix in its
    // general form, so two fused gates cost what they cost apart, plus the saved sweep)
    p.sweep_flops = !c128 ? 24.0 : (st.prec == QS_PREC_DF32 ? 8.0 : 1.0);
    // complex64 with fusion width 4..6: dense blocks go to the tensor cores (K3)
    p.tc = !c128 && o.fuse_k >= 4 && tc_available(p.m, std::min(o.fuse_k, 6));
    p.force_chunk = o.mode == QS_MODE_CHUNK;
    // complex128 single-state passes: a two-qubit diagonal with one qubit outside the local
    // set is a per-tile factor on the other (non-local terms folded into the block's table)
    p.hi_diag = c128;
    if (p.tc) {
        p.fuse_k = std::min(o.fuse_k, 6);
        p.sweep_flops = 1e30;  // fuse whenever the block fits: its cost is on the tensor pipe
    }
    return p;
}

namespace {

// One greedy pass from the first open op, local qubits restricted to low | allowed.
// Returns the ops it takes (in order) and its local mask (unpadded).
struct Trial {
    std::vector<int> ops;
    uint64_t L = 0;
    bool stream = false;
};

// What the pass builder asks of each op, computed once per plan (a plan tries many passes).
struct OpInfo {
    uint64_t qm;   // qubits
    uint64_t hi;   // qubits that may be its only local one (pp.hi_diag)
    bool diag;
    bool chunk;
};

std::vector<OpInfo> op_info(const std::vector<Op> &ops, const PlanParams &pp) {
    std::vector<OpInfo> info(ops.size());
    for (size_t i = 0; i < ops.size(); i++) {
        info[i].qm = ops[i].qmask();
        info[i].diag = op_is_diagonal(ops[i]);
        info[i].chunk = chunkable(ops[i], pp);
        info[i].hi = pp.hi_diag ? hi_local_choices(ops[i]) : 0;
    }
    return info;
}

Trial greedy_pass(const std::vector<OpInfo> &ops, const std::vector<char> &done, size_t first, int n,
                  const PlanParams &pp, uint64_t allowed) {
    const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1ull);
    const uint64_t low = (1ull << pp.c) - 1ull;
    Trial tr;
    // qubits of ops left for a later pass: a non-diagonal op left behind blocks every later
    // op on its qubits; a diagonal one only blocks later non-diagonal ops (diagonal gates
    // commute with one another, so they may pass it)
    uint64_t L = low, blocked = 0, blocked_diag = 0;
    for (size_t i = first; i < ops.size(); i++) {
        if (done[i]) continue;
        const OpInfo &op = ops[i];
        const uint64_t qm = op.qm;
        const bool diag = op.diag;
        const uint64_t blk = diag ? blocked : (blocked | blocked_diag);
        if (!op.chunk) {
            if (tr.ops.empty() && !(qm & (blocked | blocked_diag))) {
                tr.stream = true;
                tr.ops.push_back((int)i);
            }
            break;  // a non-chunkable op is a barrier for this pass
        }
        bool take = false;
        if (!(qm & blk) && (qm & ~(low | allowed)) == 0 && __builtin_popcountll(L | qm) <= pp.m) {
            L |= qm;
            tr.ops.push_back((int)i);
            take = true;
        } else if (!(qm & blk) && pp.hi_diag) {
            // a controlled phase with its control local (already, or added if it fits) and
            // the other qubit a tile constant
            const uint64_t ch = op.hi;
            uint64_t q1 = ch & L;
            if (!q1) {
                const uint64_t cand = ch & (low | allowed);
                if (cand && __builtin_popcountll(L) < pp.m) q1 = cand;
            }
            if (q1) {
                L |= q1 & (~q1 + 1ull);
                tr.ops.push_back((int)i);
                take = true;
            }
        }
        if (!take) {
            if (diag) blocked_diag |= qm;
            else blocked |= qm;
        }
        if ((blocked & all) == all) break;
    }
    tr.L = L;
    return tr;
}

}  // namespace

std::vector<Pass> make_plan(const std::vector<Op> &ops, int n, const PlanParams &pp) {
    std::vector<Pass> plan;
    const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1ull);
    const int free_slots = pp.m - pp.c;
    std::vector<char> done(ops.size(), 0);
    const std::vector<OpInfo> info = op_info(ops, pp);
    size_t first = 0;
    while (first < ops.size()) {
        while (first < ops.size() && done[first]) first++;
        if (first >= ops.size()) break;
        // candidates: unrestricted greedy, and greedy restricted to each window of
        // free_slots consecutive high qubits (chains and brickwork advance further when the
        // local window is chosen, not claimed by the first gates in circuit order)
        Trial best = greedy_pass(info, done, first, n, pp, all);
        if (!best.stream && free_slots > 0 && n > pp.m) {
            for (int s = pp.c; s + free_slots <= n; s++) {
                const uint64_t win = ((1ull << free_slots) - 1ull) << s;
                Trial t = greedy_pass(info, done, first, n, pp, win);
                if (!t.stream && t.ops.size() > best.ops.size()) best = std::move(t);
            }
        }
        Pass pass;
        pass.ops = best.ops;
        pass.stream = best.stream;
        if (pass.ops.empty()) {
            // nothing fits next to the always-local low qubits (tiny m): stream the op
            pass.stream = true;
            pass.ops.push_back((int)first);
        }
        for (int i : pass.ops) done[i] = 1;
        if (!pass.stream) {
            uint64_t L = best.L;
            // pad with the lowest free qubits (longer contiguous runs)
            for (int b = 0; b < n && __builtin_popcountll(L) < pp.m; b++) L |= 1ull << b;
            pass.lmask = L & all;
            if (pass.ops.size() == 1 && !pp.force_chunk) pass.stream = true;
        }
        plan.push_back(std::move(pass));
    }
    return plan;
}

std::vector<Pass> choose_plan(const std::vector<Op> &ops, int n, const PlanParams &pp, const qs_options &o,
                              std::vector<Op> &merged, std::vector<std::pair<size_t, size_t>> &origin) {
    // Merged diagonal runs (one phase-function pass each) help where a run reaches more
    // qubits than a chunk pass holds (QAOA cost layers); chains of local diagonals are
    // cheaper inside chunk passes (TFIM).  Both plans are built; the one with fewer passes
    // over the state is run.
    merged.clear();
    origin.clear();
    std::vector<Pass> plan = make_plan(ops, n, pp);
    if ((o.flags & QS_OPT_NO_DIAG_MERGE) != 0 || !phasefn_supported(n)) return plan;
    std::vector<std::pair<size_t, size_t>> org;
    std::vector<Op> m = merge_diagonal_runs(ops, kMinMergedRun, &org);
    if (m.size() >= ops.size()) return plan;
    // each phase function is a streaming pass of its own (not chunkable): the merged plan
    // has at least that many passes, plus one if any other op is left
    size_t n_pf = 0;
    for (const Op &op : m) n_pf += op.kind == K_PHASEFN;
    if (n_pf + (m.size() > n_pf ? 1 : 0) > plan.size()) return plan;
    std::vector<Pass> alt = make_plan(m, n, pp);
    // equal pass counts: the merged runs (one table lookup per amplitude) cost less FP64
    // work than the same gates as diagonal blocks inside chunk passes
    if (alt.size() > plan.size()) return plan;
    merged = std::move(m);
    origin = std::move(org);
    return alt;
}

std::vector<Op> pass_program(const DeviceState &st, const PlanParams &pp, const Pass &p, const std::vector<Op> &ops) {
    const int local = __builtin_popcountll(p.lmask);
    std::vector<Op> pops;
    pops.reserve(p.ops.size());
    for (int i : p.ops) pops.push_back(ops[i]);
    if (st.dtype == QS_C128) defer_hadamard_scale(pops);
    std::vector<Op> fused = fuse_ops(std::move(pops), pp.fuse_k, pp.sweep_flops, p.lmask);
    if (st.dtype == QS_C128 && st.prec == QS_PREC_FP64 && st.n - local >= 8) fused = split_one_qubit_phases(fused);
    // (complex64 register phases keep U3 whole: split into a rotation between phases, with
    // the phases joined in run members, the 33-qubit brickwork took 5.77 s against 4.77 s)
    const bool phases = st.dtype == QS_C64 && st.reg_phases && !pp.tc && rphase_applicable(local, kTileThreadBits);
    if (!phases)
        fused = merge_tile_diagonals(std::move(fused), kTileDiagQubits, st.dtype == QS_C128 ? 0.5 : 4.0,
                                     pp.hi_diag ? p.lmask : 0);
    return fused;
}

void run_planned(DeviceState &st, const std::vector<Op> &ops, const qs_options &o, qs_stats &stats) {
    const int n = st.n;
    const PlanParams pp = plan_params(st, o);
    const double B = st.dtype == QS_C128 ? 16.0 : 8.0;
    // tiny states (no 128-byte runs): plain gate by gate
    if (n < pp.c + 1 || (B * (double)(1ull << pp.c)) < 128.0) {
        for (const Op &op : ops) {
            launch_stream_op(st, op);
            stats.passes++;
            stats.bytes += stream_bytes(op, n, st.dtype);
        }
        stats.ops_after_fuse = (int64_t)ops.size();
        return;
    }
    std::vector<Op> merged;
    std::vector<std::pair<size_t, size_t>> origin;
    std::vector<Pass> plan = choose_plan(ops, n, pp, o, merged, origin);
    // Tensor Product Booster: on a |0...0> state, the prefix whose gates keep the qubits in
    // independent groups is built in one write pass, if that saves at least one pass (the
    // booster's own pass counted as one: at equal counts the rest's passes can cost more,
    // e.g. a QFT whose first target's controlled phases lose their diagonal block)
    std::vector<Op> rest;
    const std::vector<Op> *src = &ops;
    if (st.known_zero && n >= kTpbMinQubits && (o.flags & QS_OPT_NO_TPB) == 0) {
        const TpbPlan tp = tpb_find(ops, n);
        if (!tp.taken.empty()) {
            std::vector<Op> r = tpb_rest(ops, tp);
            std::vector<Op> m2;
            std::vector<std::pair<size_t, size_t>> o2;
            std::vector<Pass> p2 = choose_plan(r, n, pp, o, m2, o2);
            if (p2.size() + 1 < plan.size()) {
                tpb_execute(st, ops, tp, o, stats);
                rest = std::move(r);
                src = &rest;
                plan = std::move(p2);
                merged = std::move(m2);
                origin = std::move(o2);
            }
        }
    }
    const std::vector<Op> &ops_r = merged.empty() ? *src : merged;
    // Tensor-core blocks accumulate in FP32 inside the MMA with truncation toward zero, a
    // small systematic shrink per block.  The circuit is unitary, so the FP64 squared norm
    // before it is restored afterwards (three extra read passes and one write pass).
    const bool correct_norm = pp.tc && (o.flags & QS_OPT_NO_TC_NORM_FIX) == 0;
    if (correct_norm) {
        if (!st.dev_norms) QS_CUDA(cudaMalloc(&st.dev_norms, 2 * sizeof(double)));
        reduce_norm_async(st, st.dev_norms);
    }
    int64_t n_ops = 0;
    for (const Pass &p : plan) {
        if (p.stream) {
            for (int i : p.ops) {
                launch_stream_op(st, ops_r[i]);
                stats.bytes += stream_bytes(ops_r[i], n, st.dtype);
                n_ops++;
            }
            stats.passes++;
            continue;
        }
        const std::vector<Op> fused = pass_program(st, pp, p, ops_r);
        stats.tile_sweeps += launch_pass_ops(st, p.lmask, fused, pp.tc, &stats);
        stats.passes++;
        stats.bytes += 2.0 * B * (double)(1ull << n);
        n_ops += (int64_t)fused.size();
    }
    if (correct_norm) {
        reduce_norm_async(st, st.dev_norms + 1);
        launch_scale_ratio(st, st.dev_norms);
        stats.bytes += 4.0 * B * (double)(1ull << n);
    }
    stats.ops_after_fuse = n_ops;
}

}  // namespace qs
