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
// term counts, unscaled Hadamard runs, nothing fused across the local set), and runs the
// chunk-pass program as launched: its tile KOps (make_tile_kop, then join_h_cdiag)
// interpreted tile by tile on the CPU from the semantics kops.cuh documents; likewise the
// streaming ops of gate-by-gate and fused calls (make_kop on the whole state).  Finally the
// whole planned complex128 path (plan_params, choose_plan, pass_program) is emulated on
// 10- and 14-qubit states with several chunk widths, FP64 and double-float.
// Usage: host_transforms_check <seed> <trials>; prints OK and exits 0 on success.
//        host_transforms_check --gates; prints the lowered gate matrices.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "chunk.h"
#include "kgeom.h"
#include "phasefn.h"
#include "plan.h"
#include "qs_internal.h"
#include "tpb.h"

namespace qs {
void fail(int code, const std::string &msg) { throw Error{code, msg}; }
void cuda_check(cudaError_t, const char *what) { fail(QS_ERR_CUDA, what); }
// The planner's host code is linked as it is; everything that would touch a GPU fails.
void launch_chunk_pass(DeviceState &, uint64_t, const std::vector<KOp> &, const std::vector<double> &) {
    fail(QS_ERR_INVALID, "no GPU in this check");
}
void launch_chunk_pass_tc(DeviceState &, uint64_t, const std::vector<KOp> &, const std::vector<double> &,
                          const std::vector<float> &, uint32_t) {
    fail(QS_ERR_INVALID, "no GPU in this check");
}
void launch_stream_op(DeviceState &, const Op &) { fail(QS_ERR_INVALID, "no GPU in this check"); }
void reduce_norm_async(DeviceState &, double *) { fail(QS_ERR_INVALID, "no GPU in this check"); }
void launch_scale_ratio(DeviceState &, const double *) { fail(QS_ERR_INVALID, "no GPU in this check"); }
bool tc_available(int, int) { return false; }
void build_tc_operand(const std::vector<cd> &, int, std::vector<float> &, int &, int &) {
    fail(QS_ERR_INVALID, "no GPU in this check");
}
// states of at least 9 qubits (the phase-function pass works in units of 2^9 amplitudes)
bool phasefn_supported(int n) { return n >= 9; }
void launch_set_zero_state(DeviceState &) { fail(QS_ERR_INVALID, "no GPU in this check"); }
void launch_tpb_product(DeviceState &, const void *const *, const uint64_t *, int) {
    fail(QS_ERR_INVALID, "no GPU in this check");
}
void run_circuit(DeviceState &, const std::vector<Op> &, const qs_options &, qs_stats &) {
    fail(QS_ERR_INVALID, "no GPU in this check");
}
void free_device_state(DeviceState &) {}
void arena_reserve(DeviceState &, size_t) { fail(QS_ERR_INVALID, "no GPU in this check"); }
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

// Random unitary of dimension D (Gram-Schmidt on Gaussian columns), row-major (re, im).
std::vector<double> random_unitary(std::mt19937_64 &g, int D) {
    std::normal_distribution<double> N;
    std::vector<cd> u((size_t)D * D);
    for (int c = 0; c < D; c++) {
        std::vector<cd> v(D);
        for (cd &z : v) z = cd(N(g), N(g));
        for (int p = 0; p < c; p++) {
            cd dot = 0.0;
            for (int r = 0; r < D; r++) dot += std::conj(u[(size_t)r * D + p]) * v[r];
            for (int r = 0; r < D; r++) v[r] -= dot * u[(size_t)r * D + p];
        }
        double nrm = 0.0;
        for (const cd &z : v) nrm += std::norm(z);
        nrm = std::sqrt(nrm);
        for (int r = 0; r < D; r++) u[(size_t)r * D + c] = v[r] / nrm;
    }
    std::vector<double> out;
    for (const cd &z : u) {
        out.push_back(z.real());
        out.push_back(z.imag());
    }
    return out;
}

// Random gate records of every type (QS_DENSE: a random unitary on 1 to 3 qubits), angles
// uniform in [0, 2 pi);
// with lmask != 0 only gates a chunk pass over that local set may hold: all qubits local,
// or a two-qubit diagonal whose one local qubit may carry it (hi_local_choices).
// Mixes: 0 every type alike, 1 QFT-like (Hadamard targets with controlled phases),
// 2 Hadamard-heavy (four in five gates, runs past the unscaled limit), 3 QAOA-like
// (layers of equal-angle RZZ on random pairs or on every pair of a random qubit set,
// then RX on every qubit).
std::vector<Op> random_ops(std::mt19937_64 &g, int n, int count, uint64_t lmask, int mix) {
    std::uniform_real_distribution<double> ang(0.0, 2.0 * M_PI);
    std::vector<Op> ops;
    auto local = [&](int q) { return lmask == 0 || ((lmask >> q) & 1ull); };
    while ((int)ops.size() < count) {
        qs_gate r{};
        if (mix == 3) {  // a cost layer of RZZ (one angle per layer), then the RX mixer
            const double gamma = ang(g), beta = ang(g);
            std::vector<std::pair<int, int>> edges;
            if (g() & 1) {  // every pair of a random set of 4 to 7 qubits (fully connected)
                std::vector<int> set;
                const int w = 4 + (int)(g() % 4);
                while ((int)set.size() < w) {
                    const int q = (int)(g() % n);
                    if (std::find(set.begin(), set.end(), q) == set.end()) set.push_back(q);
                }
                for (int i = 0; i < w; i++)
                    for (int j = i + 1; j < w; j++) edges.push_back({set[i], set[j]});
            } else {  // 2n random pairs
                for (int e = 0; e < 2 * n; e++) {
                    const int a = (int)(g() % n);
                    int b;
                    do b = (int)(g() % n);
                    while (b == a);
                    edges.push_back({a, b});
                }
            }
            for (const auto &e : edges) {
                if ((int)ops.size() >= count) break;
                qs_gate z{};
                z.type = QS_RZZ;
                z.nq = 2;
                z.q[0] = e.first;
                z.q[1] = e.second;
                z.p[0] = gamma;
                if (local(z.q[0]) && local(z.q[1])) ops.push_back(lower_gate(z));
            }
            for (int q = 0; q < n && (int)ops.size() < count; q++) {
                if (!local(q)) continue;
                qs_gate x{};
                x.type = QS_RX;
                x.nq = 1;
                x.q[0] = q;
                x.p[0] = beta;
                ops.push_back(lower_gate(x));
            }
            continue;
        }
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
        r.type = (mix == 2 && g() % 5 != 0) ? QS_H : (int)(g() % 18);
        r.nq = r.type == QS_DENSE ? 1 + (int)(g() % 3) : (r.type >= QS_CNOT ? 2 : 1);
        for (int j = 0; j < r.nq; j++) {
            bool again;
            do {
                r.q[j] = (int)(g() % n);
                again = false;
                for (int i = 0; i < j; i++) again = again || r.q[i] == r.q[j];
            } while (again);
        }
        for (double &p : r.p) p = ang(g);
        std::vector<double> dense;
        if (r.type == QS_DENSE) {
            dense = random_unitary(g, 1 << r.nq);
            r.m = dense.data();
        }
        validate_gate(r, n);
        Op op = lower_gate(r);
        bool ok = true;
        for (int j = 0; j < op.k; j++) ok = ok && local(op.q[j]);
        if (!ok && op.k == 2 && r.type != QS_DENSE)
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

// fused blocks: at most fuse_k qubits (a wider gate passes through as it is)
void check_fused(const std::vector<Op> &ops, int fuse_k, int widest_gate, uint64_t lmask, int trial) {
    for (const Op &b : ops) {
        if (b.kind == K_DENSE || (b.kind == K_DIAG && b.k > 2))
            check(b.k <= std::max(fuse_k, widest_gate), "fused block wider than fuse_k", trial);
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

// ---- tile programs: the KOps a chunk pass launches, interpreted on the CPU --------------
// Each tile holds the 2^m amplitudes whose non-local qubits equal the tile's bits; tile
// position r is the r-th qubit of the local set.  Semantics per KOp kind as the kernels
// document them (kops.cuh): groups of elements base + off[t] over the bases with the fixed
// bits fb clear and set_mask set; F_DIAGK / F_DENSEK on positions pos[]; F_CDIAGK on the
// elements with its control positions set, with the factors of its terms whose global
// qubit is 1 in the tile; F_HCDIAGK the unscaled butterfly across its control first.
int g_joins = 0;

// A register phase (F_RPHASE) as the chunk kernel runs it, thread by thread: every thread
// holds the 2^kRpBits amplitudes spanned by the phase's register positions, register r
// holding the one whose register bits are r ^ sigma (sigma from the lane bits for
// positions below 4, as the kernel lays them out), and applies the members in program
// order with the same operand encoding, conjugation by sigma, exchange relabelling and
// parity counting; then stores in the final register order.  Double precision.
int g_rp_members = 0;
int g_rp_runs = 0;

void apply_rphase(State &tile, int m, const KOp &ph, const std::vector<double> &mats) {
    const int nt = ph.nt;
    const uint32_t threads = 1u << nt;
    if (m != nt + kRpBits) fail(QS_ERR_INVALID, "register phase: m != thread bits + 5");
    const double *prog = mats.data() + ph.mat;
    const uint32_t pattern[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
    for (uint32_t tid = 0; tid < threads; tid++) {
        const uint32_t lane = tid & 31u;
        // geometry: register positions, sigma, base
        uint32_t pb[kRpBits], sigma = 0, base = 0;
        int nlow = 0;
        for (int j = 0; j < kRpBits; j++) {
            pb[j] = 1u << ph.pos[j];
            nlow += ph.pos[j] < 4 ? 1 : 0;
        }
        int li = 4 - nlow;
        for (int j = 0; j < kRpBits; j++)
            if (ph.pos[j] < 4) {
                sigma |= ((lane >> li) & 1u) << j;
                li++;
            }
        for (int i = 0; i < nt; i++) base |= ((tid >> i) & 1u) << (uint32_t)((ph.off[0] >> (4 * i)) & 15u);
        const uint32_t sigma0 = sigma;
        auto index = [&](uint32_t r, uint32_t sg) {
            uint32_t o = base;
            for (int j = 0; j < kRpBits; j++)
                if (((r ^ sg) >> j) & 1u) o ^= pb[j];
            return o;
        };
        cd v[32];
        for (uint32_t r = 0; r < 32; r++) v[r] = tile[index(r, sigma0)];
        auto mask = [&](int enc) -> uint32_t {
            if (enc == kRpAlways) return 0xFFFFFFFFu;
            if (enc == kRpNever) return 0u;
            if (enc & 16) {
                const int j = enc & 15;
                return ((sigma >> j) & 1u) ? ~pattern[j] : pattern[j];
            }
            return ((tid >> enc) & 1u) ? 0xFFFFFFFFu : 0u;
        };
        auto is_slot = [](int enc) { return (enc & 16) && enc < kRpNever; };
        auto pairs = [&](int J, auto fn) {
            for (uint32_t r = 0; r < 32; r++)
                if (!((r >> J) & 1u)) fn(r, r | (1u << J));
        };
        const int nmem = (int)prog[0];
        const double *mm = prog + 1;
        for (int i = 0; i < nmem; i++) {
            g_rp_members++;
            const int code = (int)mm[0];
            const int type = code & 7, J = (code >> 3) & 7, ea = (code >> 6) & 31, eb = (code >> 11) & 31;
            const int len = (code >> 16) & 255;
            const double *P = mm + 1;
            mm += 1 + len;
            const int f = (int)((sigma >> J) & 1u);
            auto general = [&](cd (&M)[4]) {  // X M X where bit J of sigma is set
                const cd g[4] = {cd(P[0], P[1]), cd(P[2], P[3]), cd(P[4], P[5]), cd(P[6], P[7])};
                if (f) { M[0] = g[3]; M[1] = g[2]; M[2] = g[1]; M[3] = g[0]; }
                else { M[0] = g[0]; M[1] = g[1]; M[2] = g[2]; M[3] = g[3]; }
            };
            switch (type) {
            case RP_M1: {
                cd M[4];
                if (eb == RP_R0) {
                    if (f) fail(QS_ERR_INVALID, "register phase: 7-real form on a conjugated slot");
                    M[0] = P[0]; M[1] = cd(P[1], P[2]); M[2] = cd(P[3], P[4]); M[3] = cd(P[5], P[6]);
                } else if (eb == RP_REAL || eb == RP_RX) {
                    const double q0 = P[3 * f], q1 = P[1 + f], q2 = P[2 - f], q3 = P[3 - 3 * f];
                    if (eb == RP_REAL) { M[0] = q0; M[1] = q1; M[2] = q2; M[3] = q3; }
                    else { M[0] = q0; M[1] = cd(0, q1); M[2] = cd(0, q2); M[3] = q3; }
                } else {
                    general(M);
                }
                pairs(J, [&](uint32_t a, uint32_t b) {
                    const cd x = v[a], y = v[b];
                    v[a] = M[0] * x + M[1] * y;
                    v[b] = M[2] * x + M[3] * y;
                });
                break;
            }
            case RP_C1: {
                cd M[4];
                general(M);
                const uint32_t K = mask(ea);
                pairs(J, [&](uint32_t a, uint32_t b) {
                    if (!((K >> a) & 1u)) return;
                    const cd x = v[a], y = v[b];
                    v[a] = M[0] * x + M[1] * y;
                    v[b] = M[2] * x + M[3] * y;
                });
                break;
            }
            case RP_X: {
                const uint32_t K = mask(ea);
                if (K == 0u || K == 0xFFFFFFFFu) {
                    sigma ^= (K & 1u) << J;
                    break;
                }
                pairs(J, [&](uint32_t a, uint32_t b) {
                    if ((K >> a) & 1u) std::swap(v[a], v[b]);
                });
                break;
            }
            case RP_DIAG: {
                const uint32_t Ka = mask(ea), Kb = mask(eb);
                for (uint32_t r = 0; r < 32; r++) {
                    const int s = (int)(2 * ((Ka >> r) & 1u) + ((Kb >> r) & 1u));
                    v[r] *= cd(P[2 * s], P[2 * s + 1]);
                }
                break;
            }
            case RP_NEG: {
                uint32_t K = 0;
                for (int q = 0; q <= J; q++) {
                    const int e = (int)P[q];
                    K ^= mask(e & 31) & mask(e >> 5);
                }
                for (uint32_t r = 0; r < 32; r++)
                    if ((K >> r) & 1u) v[r] = -v[r];
                break;
            }
            case RP_PARITY: {
                const uint32_t K = mask(ea) ^ mask(eb);
                for (uint32_t r = 0; r < 32; r++) v[r] *= ((K >> r) & 1u) ? cd(P[2], P[3]) : cd(P[0], P[1]);
                break;
            }
            case RP_PARITYN: {
                const int np = (len - 2) / 3;
                int cnt[32] = {0};
                int slot_patterns = 0;
                for (int q = 0; q < np; q++) {
                    const int e = (int)P[q];
                    const uint32_t M = mask(e & 31) ^ mask(e >> 5);
                    slot_patterns += is_slot(e & 31) || is_slot(e >> 5);
                    for (uint32_t r = 0; r < 32; r++) cnt[r] += (int)((M >> r) & 1u);
                }
                if (slot_patterns > 15) fail(QS_ERR_INVALID, "register phase: more than 15 counted patterns");
                for (uint32_t r = 0; r < 32; r++) v[r] *= cd(P[np + 2 * cnt[r]], P[np + 2 * cnt[r] + 1]);
                break;
            }
            default: {  // RP_PH: one phase, or (slot field 1) a run of phases and sign pairs
                if (J == 1) {
                    g_rp_runs++;
                    for (int q = 0; q < ea; q++) {
                        const uint32_t K = mask((int)P[3 * q]);
                        for (uint32_t r = 0; r < 32; r++)
                            if ((K >> r) & 1u) v[r] *= cd(P[3 * q + 1], P[3 * q + 2]);
                    }
                    uint32_t K = 0;
                    for (int q = 0; q < eb; q++) {
                        const int e = (int)P[3 * ea + q];
                        K ^= mask(e & 31) & mask(e >> 5);
                    }
                    for (uint32_t r = 0; r < 32; r++)
                        if ((K >> r) & 1u) v[r] = -v[r];
                    break;
                }
                const uint32_t K = mask(ea) & mask(eb);
                for (uint32_t r = 0; r < 32; r++)
                    if ((K >> r) & 1u) v[r] *= cd(P[0], P[1]);
                break;
            }
            }
        }
        for (uint32_t r = 0; r < 32; r++) tile[index(r, sigma)] = v[r];
    }
}

void apply_kop(State &tile, int m, const KOp &k, const std::vector<double> &mats, uint64_t base) {
    auto C = [&](int i) { return cd(mats[(size_t)k.mat + 2 * i], mats[(size_t)k.mat + 2 * i + 1]); };
    const uint32_t N = 1u << m;
    auto table_index = [&](uint32_t x, int kt) {
        uint32_t s = 0;
        for (int j = 0; j < kt; j++) s |= ((x >> k.pos[j]) & 1u) << (kt - 1 - j);
        return s;
    };
    switch (k.fkind) {
    case F_DIAGK:
        for (uint32_t x = 0; x < N; x++) tile[x] *= C((int)table_index(x, k.k));
        return;
    case F_CDIAGK:
    case F_HCDIAGK: {
        uint32_t cm = 0;
        for (int j = 0; j < k.nf; j++) cm |= 1u << k.pos[k.k + j];
        if (cm != (uint32_t)k.set_mask) fail(QS_ERR_INVALID, "controls and set_mask disagree");
        if (k.fkind == F_HCDIAGK && k.nf != 1) fail(QS_ERR_INVALID, "joined block with several controls");
        const int ne = 1 << k.k;
        for (uint32_t x = 0; x < N; x++) {
            if ((x & cm) != cm) continue;
            const uint32_t s = table_index(x, k.k);
            cd f = C((int)s);
            for (int i = 0; i < k.nt; i++) {
                const double *t = &mats[(size_t)k.mat + 2 * ne + 4 * i];
                const int tb = (int)t[0], h = (int)t[1];
                if (((base >> h) & 1ull) && (tb < 0 || ((s >> tb) & 1u))) f *= cd(t[2], t[3]);
            }
            if (k.fkind == F_HCDIAGK) {
                const uint32_t x0 = x ^ (1u << k.pos[k.k]);
                const cd a0 = tile[x0], a1 = tile[x];
                tile[x0] = a0 + a1;
                tile[x] = (a0 - a1) * f;
            } else {
                tile[x] *= f;
            }
        }
        return;
    }
    case F_DENSEK: {
        const uint32_t D = 1u << k.k;
        uint32_t pm = 0;
        for (int j = 0; j < k.k; j++) pm |= 1u << k.pos[j];
        std::vector<cd> in(D);
        std::vector<uint32_t> idx(D);
        for (uint32_t b = 0; b < N; b++) {
            if (b & pm) continue;
            for (uint32_t v = 0; v < D; v++) {
                uint32_t e = b;
                for (int j = 0; j < k.k; j++)
                    if ((v >> (k.k - 1 - j)) & 1u) e |= 1u << k.pos[j];
                idx[v] = e;
                in[v] = tile[e];
            }
            for (uint32_t r = 0; r < D; r++) {
                cd acc = 0.0;
                for (uint32_t c = 0; c < D; c++) acc += C((int)(r * D + c)) * in[c];
                tile[idx[r]] = acc;
            }
        }
        return;
    }
    default:
        break;
    }
    int nt;
    switch (k.fkind) {
    case F_PHASE: case F_NEG: nt = 1; break;
    case F_H: case F_SWAP: case F_DIAG1: case F_DENSE1: nt = 2; break;
    case F_DIAG2: case F_DENSE2: nt = 4; break;
    case F_RPHASE: apply_rphase(tile, m, k, mats); return;
    default: fail(QS_ERR_INVALID, "tile op kind outside this check");
    }
    uint32_t fm = 0;
    for (int j = 0; j < k.nf; j++) fm |= 1u << k.fb[j];
    for (uint32_t x = 0; x < N; x++) {
        if (x & fm) continue;
        const uint32_t b = x | (uint32_t)k.set_mask;
        uint32_t e[4];
        cd a[4];
        for (int t = 0; t < nt; t++) {
            e[t] = b + (uint32_t)k.off[t];
            a[t] = tile[e[t]];
        }
        cd o[4];
        switch (k.fkind) {
        case F_PHASE: o[0] = a[0] * C(0); break;
        case F_NEG: o[0] = -a[0]; break;
        case F_H: {
            const double r = k.nmat >= 1 ? mats[(size_t)k.mat] : 1.0 / std::sqrt(2.0);
            o[0] = r * (a[0] + a[1]);
            o[1] = r * (a[0] - a[1]);
            break;
        }
        case F_SWAP: o[0] = a[1]; o[1] = a[0]; break;
        case F_DIAG1: o[0] = a[0] * C(0); o[1] = a[1] * C(1); break;
        case F_DIAG2:
            for (int t = 0; t < 4; t++) o[t] = a[t] * C(t);
            break;
        default:  // F_DENSE1, F_DENSE2: the full matrix, row-major
            for (int r = 0; r < nt; r++) {
                o[r] = 0.0;
                for (int c = 0; c < nt; c++) o[r] += C(r * nt + c) * a[c];
            }
        }
        for (int t = 0; t < nt; t++) tile[e[t]] = o[t];
    }
}

State run_tiles(const State &psi0, int n, uint64_t L, const std::vector<KOp> &kops, const std::vector<double> &mats) {
    std::vector<int> lq, hq;
    for (int b = 0; b < n; b++) ((L >> b) & 1ull ? lq : hq).push_back(b);
    const int m = (int)lq.size();
    State psi = psi0, tile((size_t)1 << m);
    for (uint64_t t = 0; t < (1ull << hq.size()); t++) {
        uint64_t base = 0;
        for (size_t j = 0; j < hq.size(); j++)
            if ((t >> j) & 1ull) base |= 1ull << hq[j];
        auto gidx = [&](uint32_t x) {
            uint64_t a = base;
            for (int r = 0; r < m; r++)
                if ((x >> r) & 1u) a |= 1ull << lq[r];
            return a;
        };
        for (uint32_t x = 0; x < tile.size(); x++) tile[x] = psi[gidx(x)];
        for (const KOp &k : kops) apply_kop(tile, m, k, mats, base);
        for (uint32_t x = 0; x < tile.size(); x++) psi[gidx(x)] = tile[x];
    }
    return psi;
}

// The pass program as launched: tile KOps on tile-local positions, then the Hadamard join.
void check_tile_program(const State &psi0, const State &ref, int n, uint64_t lmask, const std::vector<Op> &prog,
                        double tol, int trial) {
    const uint64_t L = lmask ? lmask : (1ull << n) - 1;
    int pos[64] = {0};
    int r = 0;
    for (int b = 0; b < n; b++)
        if ((L >> b) & 1ull) pos[b] = r++;
    std::vector<double> mats;
    std::vector<KOp> kops;
    for (const Op &op : prog) kops.push_back(make_tile_kop(op, pos, mats));
    check(rel_err(ref, run_tiles(psi0, n, L, kops, mats)) < tol, "tile program", trial);
    const std::vector<KOp> joined = join_h_cdiag(kops, mats);
    for (const KOp &k : joined) g_joins += k.fkind == F_HCDIAGK;
    check(rel_err(ref, run_tiles(psi0, n, L, joined, mats)) < tol, "tile program with joined Hadamards", trial);
}

// Streaming ops (one pass over the whole state each): make_kop on the state's own bit
// positions, interpreted with the whole state as one tile.
void check_stream_program(const State &psi0, const State &ref, int n, const std::vector<Op> &prog, const char *what,
                          double tol, int trial) {
    int ident[64];
    for (int i = 0; i < 64; i++) ident[i] = i;
    std::vector<double> mats;
    std::vector<KOp> kops;
    for (const Op &op : prog) kops.push_back(make_kop(op, ident, mats));
    check(rel_err(ref, run_tiles(psi0, n, (1ull << n) - 1, kops, mats)) < tol, what, trial);
}

// A merged diagonal run (K_PHASEFN) as phasefn.h defines it: F(x) = table[sum over groups of
// count_g(x) * stride_g], count = popcount(x & mask) (PF_WEIGHT) or the number of pairs with
// both bits set (PF_PAIRS).
void apply_phasefn(State &psi, const Op &op) {
    const PhaseFn &f = *op.pf;
    for (size_t x = 0; x < psi.size(); x++) {
        size_t idx = 0;
        for (const PfGroup &gr : f.groups) {
            int count = 0;
            if (gr.kind == PF_WEIGHT) {
                count = __builtin_popcountll((uint64_t)x & gr.mask);
            } else {
                for (const auto &pr : gr.pairs) count += ((x >> pr.first) & 1) && ((x >> pr.second) & 1);
            }
            idx += (size_t)count * (size_t)gr.stride;
        }
        psi[x] *= f.table.at(idx);
    }
}

// A complex128 call of the planned path, emulated: the real planner (choose_plan, merged
// diagonal runs included) and per-pass program (pass_program); streaming passes apply
// their ops directly, chunk passes run their tile programs as launched.  Every op must
// run exactly once, every chunk pass must keep the low c qubits local, and the result
// must equal the gates applied one by one.
int g_planned_passes = 0, g_planned_terms = 0, g_phasefns = 0;

void check_planned(const State &psi0, const State &ref, int n, const std::vector<Op> &ops, int chunk_m, int prec,
                   int mode, double tol, int trial, int dtype = QS_C128, bool reg_phases = false) {
    DeviceState st;
    st.n = n;
    st.dtype = dtype;
    st.prec = prec;
    st.reg_phases = reg_phases;  // complex64: register phases, or one shared-memory sweep per op
    qs_options o{};
    o.mode = mode;
    o.chunk_m = chunk_m;
    o.precision = prec;
    const PlanParams pp = plan_params(st, o);
    std::vector<Op> merged;
    std::vector<std::pair<size_t, size_t>> origin;
    const std::vector<Pass> plan = choose_plan(ops, n, pp, o, merged, origin);
    const std::vector<Op> &ops_r = merged.empty() ? ops : merged;
    std::vector<int> seen(ops_r.size(), 0);
    State psi = psi0;
    for (const Pass &p : plan) {
        g_planned_passes++;
        for (int i : p.ops) seen[(size_t)i]++;
        if (p.stream) {
            for (int i : p.ops) {
                if (ops_r[(size_t)i].kind == K_PHASEFN) {
                    apply_phasefn(psi, ops_r[(size_t)i]);
                    g_phasefns++;
                }
                else apply(psi, ops_r[(size_t)i]);
            }
            continue;
        }
        const uint64_t low = (1ull << pp.c) - 1ull;
        check((p.lmask & low) == low, "chunk pass without the low qubits", trial);
        check(__builtin_popcountll(p.lmask) <= pp.m, "chunk pass wider than m", trial);
        const std::vector<Op> prog = pass_program(st, pp, p, ops_r);
        int pos[64] = {0};
        int r = 0;
        for (int b = 0; b < n; b++)
            if ((p.lmask >> b) & 1ull) pos[b] = r++;
        std::vector<double> mats;
        std::vector<KOp> kops;
        if (dtype == QS_C64 && reg_phases && rphase_applicable(r, kTileThreadBits)) {
            // the register-phase programs launch_pass_ops builds for complex64 tiles
            kops = build_register_phases(prog, pos, r, kTileThreadBits, mats);
        } else {
            for (const Op &op : prog) {
                kops.push_back(make_tile_kop(op, pos, mats));
                g_planned_terms += (int)op.hi.size();
            }
        }
        if (dtype == QS_C128 && prec == QS_PREC_FP64) kops = join_h_cdiag(kops, mats);
        psi = run_tiles(psi, n, p.lmask, kops, mats);
    }
    for (int c : seen) check(c == 1, "op not run exactly once", trial);
    check(rel_err(ref, psi) < tol, reg_phases ? "planned path (register phases)" : "planned path", trial);
}

}  // namespace

// --gates: each fixed gate type lowered (lower_gate) at a few angle sets, as lines
// "type p0 p1 p2 k re im re im ..." of its full 2^k x 2^k matrix (first operand most
// significant), for a comparison with the oracle's own gate matrices.
int print_lowered_gates() {
    const double sets[][3] = {{0.0, 0.0, 0.0}, {M_PI, M_PI / 2, -M_PI / 4}, {0.3, 1.7, -2.9}, {5.1, -0.4, 2.2}};
    for (int type = 0; type < QS_DENSE; type++) {
        for (const auto &ps : sets) {
            qs_gate r{};
            r.type = type;
            r.nq = type >= QS_CNOT ? 2 : 1;
            r.q[0] = 0;
            r.q[1] = 1;
            for (int j = 0; j < 3; j++) r.p[j] = ps[j];
            const Op op = lower_gate(r);
            const std::vector<cd> f = op.full();
            std::printf("%d %.17g %.17g %.17g %d", type, ps[0], ps[1], ps[2], op.k);
            for (const cd &z : f) std::printf(" %.17g %.17g", z.real(), z.imag());
            std::printf("\n");
        }
    }
    return 0;
}

// Tensor Product Booster host logic: on |0...0>, the prefix tpb_find takes, built as the
// tensor product of the groups' sub-states (each from its relabelled ops, tpb_group_ops),
// followed by the ops it leaves (tpb_rest), must give the circuit's state; the plan must
// keep its limits (components, groups) and take no op that shares a qubit with an earlier
// op left out.
int g_tpb_taken = 0;

void check_tpb(std::mt19937_64 &g, int n, int mix, double tol, int trial) {
    std::uniform_real_distribution<double> ang(0.0, 2.0 * M_PI);
    std::vector<Op> ops;
    // a product-friendly start: one-qubit layer, then gates on neighbouring pairs
    for (int q = 0; q < n; q++) {
        qs_gate r{};
        r.type = (trial & 1) ? QS_H : QS_U3;
        r.nq = 1;
        r.q[0] = q;
        for (double &p : r.p) p = ang(g);
        ops.push_back(lower_gate(r));
    }
    for (int e = 0; e < n; e++) {
        qs_gate r{};
        const int types[4] = {QS_CZ, QS_CNOT, QS_RZZ, QS_CU3};
        r.type = types[g() % 4];
        r.nq = 2;
        r.q[0] = (int)(g() % n);
        r.q[1] = (r.q[0] + 1 + (int)(g() % 2)) % n;
        for (double &p : r.p) p = ang(g);
        ops.push_back(lower_gate(r));
    }
    const std::vector<Op> tail = random_ops(g, n, 40, 0, mix);
    ops.insert(ops.end(), tail.begin(), tail.end());
    State zero((size_t)1 << n, 0.0);
    zero[0] = 1.0;
    const State ref = run(zero, ops);
    const uint64_t all = (1ull << n) - 1ull;
    for (const auto &lim : std::vector<std::pair<int, int>>{{1, 3}, {2, 4}, {3, 5}, {4, 6}, {14, 17}}) {
        const TpbPlan tp = tpb_find(ops, n, lim.first, lim.second);
        if (tp.taken.empty()) continue;
        g_tpb_taken += (int)tp.taken.size();
        uint64_t cover = 0;
        bool ok = (int)tp.group_mask.size() <= kTpbMaxGroups && tp.group_ops.size() == tp.group_mask.size();
        for (uint64_t gm : tp.group_mask) {
            ok &= (cover & gm) == 0 && __builtin_popcountll(gm) <= lim.second;
            cover |= gm;
        }
        check(ok && cover == all, "booster groups do not partition the qubits within their limit", trial);
        std::vector<char> taken(ops.size(), 0);
        for (int i : tp.taken) taken[i] = 1;
        uint64_t left = 0;
        int comp[64];
        for (int q = 0; q < n; q++) comp[q] = q;
        for (size_t i = 0; i < ops.size(); i++) {
            const uint64_t qm = ops[i].qmask();
            if (!taken[i]) {
                left |= qm;
                continue;
            }
            check((qm & left) == 0, "booster took an op past an earlier op it left out", trial);
            int within = 0;
            for (uint64_t gm : tp.group_mask) within += (qm & gm) == qm;
            check(within == 1, "booster op spans groups", trial);
            const int c0 = comp[ops[i].q[0]];
            for (int j = 1; j < ops[i].k; j++) {
                const int cj = comp[ops[i].q[j]];
                for (int q = 0; q < n; q++)
                    if (comp[q] == cj) comp[q] = c0;
            }
        }
        for (int q = 0; q < n; q++) {
            int sz = 0;
            for (int p = 0; p < n; p++) sz += comp[p] == comp[q];
            check(sz <= lim.first, "booster component above its limit", trial);
        }
        // the product state, then the rest
        std::vector<State> subs;
        for (size_t gi = 0; gi < tp.group_mask.size(); gi++) {
            State s0((size_t)1 << __builtin_popcountll(tp.group_mask[gi]), 0.0);
            s0[0] = 1.0;
            subs.push_back(run(s0, tpb_group_ops(ops, tp, (int)gi, n)));
        }
        State psi((size_t)1 << n);
        for (uint64_t x = 0; x <= all; x++) {
            cd a = 1.0;
            for (size_t gi = 0; gi < subs.size(); gi++) {
                uint64_t idx = 0, m = tp.group_mask[gi];
                for (int o = 0; m; o++, m &= m - 1) idx |= ((x >> __builtin_ctzll(m)) & 1ull) << o;
                a *= subs[gi][idx];
            }
            psi[x] = a;
        }
        check(rel_err(ref, run(psi, tpb_rest(ops, tp))) < tol, "tensor-product prefix + rest", trial);
    }
}

int main(int argc, char **argv) {
    if (argc > 1 && std::string(argv[1]) == "--gates") return print_lowered_gates();
    const int seed = argc > 1 ? std::atoi(argv[1]) : 1;
    const int trials = argc > 2 ? std::atoi(argv[2]) : 20;
    std::mt19937_64 g((uint64_t)seed);
    std::normal_distribution<double> N;
    const double tol = 1e-12;
    const int n = 10;
    for (int trial = 0; trial < trials; trial++) {
        State psi0(1ull << n);
        for (cd &z : psi0) z = cd(N(g), N(g));
        // a local set of 7 of the 10 qubits (always the low 2), or none; every mix gets both
        uint64_t lmask = 0;
        if ((trial >> 2) & 1) {
            lmask = 3;
            while (__builtin_popcountll(lmask) < 7) lmask |= 1ull << (2 + g() % (n - 2));
        }
        const int mix = trial % 4;
        const std::vector<Op> ops = random_ops(g, n, mix == 2 ? 200 : 120, lmask, mix);
        const State ref = run(psi0, ops);
        int widest = 0;
        for (const Op &op : ops) widest = std::max(widest, op.k);
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
                    check_fused(f, k, widest, lmask, trial);
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
            check_tile_program(psi0, ref, n, lmask, p, tol, trial);
            if (!lmask) {
                // gate-by-gate calls (QS_MODE_GATE): global phases folded, complex128 FP64
                // Hadamards unscaled but for every 64th and the last, one streaming op each
                std::vector<Op> gops = fold_global_phases(ops);
                check_stream_program(psi0, ref, n, gops, "gate-by-gate ops", tol, trial);
                defer_hadamard_scale(gops);
                check_stream_program(psi0, ref, n, gops, "gate-by-gate ops, deferred scale", tol, trial);
                // fused calls (QS_MODE_FUSED): dense blocks of up to 3 and 6 qubits
                for (int k : {3, 6})
                    check_stream_program(psi0, ref, n, fuse_ops(ops, k), "fused blocks", tol, trial);
                // the whole planned path on this circuit: chunk widths that leave 2 to 6
                // qubits outside the tile, FP64 and double-float, auto and chunk modes
                for (int cm : {4, 6, 8})
                    for (int prec : {QS_PREC_FP64, QS_PREC_DF32})
                        check_planned(psi0, ref, n, ops, cm, prec, trial % 4 == 0 ? QS_MODE_CHUNK : QS_MODE_AUTO,
                                      tol, trial);
                // complex64 host logic (its own fusion and merge thresholds, no non-local
                // terms), applied here in double precision
                for (int cm : {5, 8})
                    check_planned(psi0, ref, n, ops, cm, QS_PREC_FP64, QS_MODE_AUTO, tol, trial, QS_C64);
            }
            if (trial % 4 == 0) {
                // 14 qubits, 6-qubit tiles: passes of 256 tiles, where complex128 FP64 splits U3
                const int n2 = 14;
                State q0((size_t)1 << n2);
                for (cd &z : q0) z = cd(N(g), N(g));
                const std::vector<Op> ops2 = random_ops(g, n2, 100, 0, (trial / 4) % 4);
                const State ref2 = run(q0, ops2);
                for (int prec : {QS_PREC_FP64, QS_PREC_DF32})
                    check_planned(q0, ref2, n2, ops2, 6, prec, QS_MODE_AUTO, tol, trial);
                // complex64 register phases: tiles of 2^13 amplitudes (256 threads x 32
                // registers), the phase programs interpreted thread by thread
                check_planned(q0, ref2, n2, ops2, 13, QS_PREC_FP64, QS_MODE_AUTO, tol, trial, QS_C64, true);
                // layers of one-qubit phases (P, S, T) with CZ and U3: runs of phases
                std::vector<Op> ph;
                std::uniform_real_distribution<double> ang(0.0, 2.0 * M_PI);
                for (int layer = 0; layer < 6; layer++) {
                    for (int q = 0; q < n2; q++) {
                        qs_gate r{};
                        r.type = (q % 3 == 0) ? QS_S : (q % 3 == 1) ? QS_T : QS_P;
                        r.nq = 1;
                        r.q[0] = q;
                        r.p[0] = ang(g);
                        ph.push_back(lower_gate(r));
                    }
                    for (int a = layer % 2; a + 1 < n2; a += 2) {
                        qs_gate r{};
                        r.type = QS_CZ;
                        r.nq = 2;
                        r.q[0] = a;
                        r.q[1] = a + 1;
                        ph.push_back(lower_gate(r));
                    }
                    for (int q = 0; q < n2; q++) {
                        qs_gate r{};
                        r.type = QS_U3;
                        r.nq = 1;
                        r.q[0] = q;
                        for (double &p : r.p) p = ang(g);
                        ph.push_back(lower_gate(r));
                    }
                }
                const State ref3 = run(q0, ph);
                check_planned(q0, ref3, n2, ph, 13, QS_PREC_FP64, QS_MODE_AUTO, tol, trial, QS_C64, true);
            }
            check_tpb(g, n, mix, tol, trial);
        } catch (const Error &e) {
            std::printf("FAIL trial %d: error %d %s\n", trial, e.code, e.msg.c_str());
            g_bad++;
        }
    }
    if (trials >= 2) check(g_tpb_taken > 0, "booster never took an op", -1);
    if (trials >= 4) check(g_rp_members > 0, "no register phase interpreted", -1);
    if (trials >= 4) check(g_rp_runs > 0, "no run of phases interpreted", -1);
    // QFT-like circuits must have exercised the join
    if (trials >= 2) check(g_joins > 0, "no Hadamard joined with its controlled block", -1);
        if (trials >= 4) check(g_planned_terms > 0 && g_phasefns > 0, "planned path not exercised", -1);
    std::printf("%s (%d trials, %d joined Hadamards, %d planned passes, %d non-local terms, %d phase functions, "
                "%d booster ops, %d register-phase members, %d phase runs)\n",
                g_bad ? "FAIL" : "OK", trials, g_joins, g_planned_passes, g_planned_terms, g_phasefns, g_tpb_taken,
                g_rp_members, g_rp_runs);
    return g_bad ? 1 : 0;
}
