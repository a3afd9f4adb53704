// Test program (built and run by tests/test_host_transforms_cpu.py, CPU only): the host
// rewrites the executor applies to a gate list before its kernels run must leave the
// circuit's action unchanged.  Each rewrite is applied to seeded random circuits on a
// small state and both op lists are applied by the plain dense loop below (each op's
// matrix on its operands, HiTerm factors where their global qubit is 1); the states must
// agree to 1e-12 of the largest amplitude.  Rewrites (Sec. II-B gate fusion and the
// executor's exact forms):
//   fold_global_phases, defer_hadamard_scale, fuse_ops (with and without a local set),
//   split_one_qubit_phases, merge_tile_diagonals (with non-local controlled phases),
//   and the chunk-pass order: deferred scale, fusion, split, diagonal merge.
// Also checks the structural limits the kernels rely on (operand counts, table sizes,
// term counts, unscaled Hadamard runs, nothing fused across the local set).
// Usage: host_transforms_check <seed> <trials>; prints OK and exits 0 on success.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "qs_internal.h"

namespace qs {
void fail(int code, const std::string &msg) { throw Error{code, msg}; }
}  // namespace qs

using namespace qs;
using State = std::vector<cd>;

namespace {

int g_bad = 0;

void check(bool ok, const char *what, int trial) {
    if (!ok) {
        std::printf("FAIL trial %d: %s\n", trial, what);
        g_bad++;
    }
}

void apply(State &psi, const Op &op) {
    const int k = op.k;
    const size_t D = 1ull << k;
    if (op.kind == K_DIAG && !op.hi.empty()) {
        for (size_t a = 0; a < psi.size(); a++) {
            size_t x = 0;
            for (int j = 0; j < k; j++) x |= ((a >> op.q[j]) & 1ull) << (k - 1 - j);
            cd f = op.m[x];
            for (const HiTerm &t : op.hi)
                if (((a >> t.h) & 1ull) && (t.t < 0 || ((a >> t.t) & 1ull))) f *= t.f;
            psi[a] *= f;
        }
        return;
    }
    const std::vector<cd> U = op.full();
    uint64_t mask = 0;
    for (int j = 0; j < k; j++) mask |= 1ull << op.q[j];
    std::vector<cd> in(D), out(D);
    std::vector<size_t> idx(D);
    for (size_t b = 0; b < psi.size(); b++) {
        if (b & mask) continue;
        for (size_t x = 0; x < D; x++) {
            size_t a = b;
            for (int j = 0; j < k; j++)
                if ((x >> (k - 1 - j)) & 1) a |= 1ull << op.q[j];
            idx[x] = a;
            in[x] = psi[a];
        }
        for (size_t r = 0; r < D; r++) {
            out[r] = 0.0;
            for (size_t c = 0; c < D; c++) out[r] += U[r * D + c] * in[c];
        }
        for (size_t x = 0; x < D; x++) psi[idx[x]] = out[x];
    }
}

State run(const State &psi0, const std::vector<Op> &ops) {
    State psi = psi0;
    for (const Op &op : ops) apply(psi, op);
    return psi;
}

double rel_err(const State &a, const State &b) {
    double e = 0.0, s = 0.0;
    for (size_t i = 0; i < a.size(); i++) {
        e = std::max(e, std::abs(a[i] - b[i]));
        s = std::max(s, std::abs(a[i]));
    }
    return e / s;
}

// Random gate records of every fixed type (no QS_DENSE), angles uniform in [0, 2 pi);
// with lmask != 0 only gates a chunk pass over that local set may hold: all qubits local,
// or a two-qubit diagonal whose one local qubit may carry it (hi_local_choices).
// Mixes: 0 every type alike, 1 QFT-like (Hadamard targets with controlled phases),
// 2 Hadamard-heavy (four in five gates, runs past the unscaled limit).
std::vector<Op> random_ops(std::mt19937_64 &g, int n, int count, uint64_t lmask, int mix) {
    std::uniform_real_distribution<double> ang(0.0, 2.0 * M_PI);
    std::vector<Op> ops;
    auto local = [&](int q) { return lmask == 0 || ((lmask >> q) & 1ull); };
    while ((int)ops.size() < count) {
        qs_gate r{};
        if (mix == 1) {  // Hadamard targets with controlled phases to every other qubit
            const int t = (int)(g() % n);
            if (!local(t)) continue;
            r.type = QS_H;
            r.nq = 1;
            r.q[0] = t;
            ops.push_back(lower_gate(r));
            for (int j = 0; j < n && (int)ops.size() < count; j++) {
                if (j == t) continue;
                qs_gate c{};
                c.type = QS_CP;
                c.nq = 2;
                const bool t_first = g() & 1;
                c.q[0] = t_first ? t : j;
                c.q[1] = t_first ? j : t;
                c.p[0] = ang(g);
                Op op = lower_gate(c);
                if (!local(j) && !((hi_local_choices(op) >> t) & 1ull)) continue;
                ops.push_back(op);
            }
            continue;
        }
        r.type = (mix == 2 && g() % 5 != 0) ? QS_H : (int)(g() % 17);
        const bool two = r.type >= QS_CNOT;
        r.nq = two ? 2 : 1;
        r.q[0] = (int)(g() % n);
        if (two) {
            do r.q[1] = (int)(g() % n);
            while (r.q[1] == r.q[0]);
        }
        for (double &p : r.p) p = ang(g);
        Op op = lower_gate(r);
        bool ok = true;
        for (int j = 0; j < op.k; j++) ok = ok && local(op.q[j]);
        if (!ok && op.k == 2)
            for (int j = 0; j < 2; j++)
                if (local(op.q[j]) && !local(op.q[1 - j]) && ((hi_local_choices(op) >> op.q[j]) & 1ull)) ok = true;
        if (ok) ops.push_back(op);
    }
    return ops;
}

int control_count(const Op &b) {
    int nctl = 0;
    for (int j = 0; j < b.k; j++) {
        const int bit = b.k - 1 - j;
        bool c = true;
        for (size_t x = 0; x < b.m.size() && c; x++)
            if (!((x >> bit) & 1) && b.m[x] != cd(1.0)) c = false;
        for (const HiTerm &t : b.hi) c = c && t.t == b.q[j];
        nctl += c;
    }
    return nctl;
}

void check_merged(const std::vector<Op> &ops, int max_k, uint64_t lmask, int trial) {
    for (const Op &b : ops) {
        if (lmask && b.hi.empty()) {
            bool all_local = (b.qmask() & ~lmask) == 0;
            check(all_local, "op with a non-local qubit and no terms", trial);
        }
        if (b.kind != K_DIAG) continue;
        check(b.k <= max_k, "diagonal block wider than max_k", trial);
        const int table_bits = b.k - control_count(b);
        check(table_bits <= (b.hi.empty() ? max_k : max_k - 1), "diagonal table too large", trial);
        check(b.hi.size() <= (size_t)kMaxHiTerms, "too many terms", trial);
        for (const HiTerm &t : b.hi) check(lmask && !((lmask >> t.h) & 1ull), "term on a local qubit", trial);
    }
}

void check_fused(const std::vector<Op> &ops, int fuse_k, uint64_t lmask, int trial) {
    for (const Op &b : ops) {
        if (b.kind == K_DENSE || (b.kind == K_DIAG && b.k > 2))
            check(b.k <= fuse_k, "fused block wider than fuse_k", trial);
        if (lmask && b.k > 2) check((b.qmask() & ~lmask) == 0, "fused across the local set", trial);
    }
}

void check_h_runs(const std::vector<Op> &ops, int trial) {
    int unscaled = 0, last = -1;
    for (size_t i = 0; i < ops.size(); i++)
        if (ops[i].kind == K_H) last = (int)i;
    for (int i = 0; i <= last; i++) {
        if (ops[i].kind != K_H) continue;
        check(!ops[i].m.empty(), "Hadamard without a scale entry", trial);
        if (ops[i].m.empty()) continue;
        if (ops[i].m[0] == cd(1.0)) {
            unscaled++;
            check(unscaled <= kMaxUnscaledH, "unscaled Hadamard run too long", trial);
        } else {
            unscaled = 0;
        }
    }
    check(last < 0 || (!ops[last].m.empty() && ops[last].m[0] != cd(1.0)), "last Hadamard unscaled", trial);
}

}  // namespace

int main(int argc, char **argv) {
    const int seed = argc > 1 ? std::atoi(argv[1]) : 1;
    const int trials = argc > 2 ? std::atoi(argv[2]) : 20;
    std::mt19937_64 g((uint64_t)seed);
    std::normal_distribution<double> N;
    const double tol = 1e-12;
    const int n = 10;
    for (int trial = 0; trial < trials; trial++) {
        State psi0(1ull << n);
        for (cd &z : psi0) z = cd(N(g), N(g));
        // a local set of 7 of the 10 qubits (always the low 2), or none
        uint64_t lmask = 0;
        if (trial % 2) {
            lmask = 3;
            while (__builtin_popcountll(lmask) < 7) lmask |= 1ull << (2 + g() % (n - 2));
        }
        const int mix = trial % 3;
        const std::vector<Op> ops = random_ops(g, n, mix == 2 ? 200 : 120, lmask, mix);
        const State ref = run(psi0, ops);
        try {
            if (!lmask) {
                check(rel_err(ref, run(psi0, fold_global_phases(ops))) < tol, "fold_global_phases", trial);
            }
            std::vector<Op> h = ops;
            defer_hadamard_scale(h);
            check_h_runs(h, trial);
            check(rel_err(ref, run(psi0, h)) < tol, "defer_hadamard_scale", trial);
            for (int k : {2, 3, 4}) {
                for (double cost : {-1.0, 1.0, 24.0}) {
                    const std::vector<Op> f = fuse_ops(ops, k, cost, lmask);
                    check_fused(f, k, lmask, trial);
                    check(rel_err(ref, run(psi0, f)) < tol, "fuse_ops", trial);
                }
            }
            check(rel_err(ref, run(psi0, split_one_qubit_phases(ops))) < tol, "split_one_qubit_phases", trial);
            for (int max_k : {3, 5, 8}) {
                const std::vector<Op> mg = merge_tile_diagonals(ops, max_k, 0.5, lmask);
                check_merged(mg, max_k, lmask, trial);
                check(rel_err(ref, run(psi0, mg)) < tol, "merge_tile_diagonals", trial);
            }
            // the order of a complex128 FP64 chunk pass
            std::vector<Op> p = ops;
            defer_hadamard_scale(p);
            p = fuse_ops(p, 4, 1.0, lmask);
            p = split_one_qubit_phases(p);
            p = merge_tile_diagonals(p, 8, 0.5, lmask);
            check_merged(p, 8, lmask, trial);
            check(rel_err(ref, run(psi0, p)) < tol, "chunk-pass pipeline", trial);
        } catch (const Error &e) {
            std::printf("FAIL trial %d: error %d %s\n", trial, e.code, e.msg.c_str());
            g_bad++;
        }
    }
    std::printf("%s (%d trials)\n", g_bad ? "FAIL" : "OK", trials);
    return g_bad ? 1 : 0;
}
