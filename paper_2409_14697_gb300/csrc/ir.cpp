// Host gate IR: validation, lowering of gate records to Ops, fusion.
//
// Gate semantics follow QueenV2 (arXiv 2409.14697) Sec. II-A: Eq. 2 (one-qubit pair
// update), Eq. 3 (CNOT on a group of four, first operand = control) and the k-qubit
// generalisation stated before Eq. 3.  The paper prints no other gate matrix; the ones
// below are the standard definitions listed in include/qs.h.  Sec. III-B notes that
// further gates are built from supported unitaries: QS_DENSE carries any such block.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "kops.cuh"
#include "qs_internal.h"

namespace qs {

namespace {

const cd kI(0.0, 1.0);

int expected_arity(int type) {
    switch (type) {
    case QS_H: case QS_X: case QS_Y: case QS_Z: case QS_S: case QS_T:
    case QS_RX: case QS_RY: case QS_RZ: case QS_P: case QS_U3:
        return 1;
    case QS_CNOT: case QS_CZ: case QS_SWAP: case QS_CU3: case QS_CP: case QS_RZZ:
        return 2;
    case QS_DENSE:
        return 0;
    default:
        return -1;
    }
}

// U3(theta, phi, lambda), OpenQASM 2 convention, row-major.
std::vector<cd> u3(double t, double p, double l) {
    const double c = std::cos(0.5 * t), s = std::sin(0.5 * t);
    return {cd(c, 0.0), -std::polar(1.0, l) * s, std::polar(1.0, p) * s,
            std::polar(1.0, p + l) * c};
}

}  // namespace

void validate_gate(const qs_gate &g, int n) {
    const int want = expected_arity(g.type);
    if (want < 0) fail(QS_ERR_INVALID, "unknown gate type " + std::to_string(g.type));
    if (want == 0) {
        if (g.nq < 1 || g.nq > 6) fail(QS_ERR_INVALID, "dense gate needs 1 <= nq <= 6");
        if (!g.m) fail(QS_ERR_INVALID, "dense gate without matrix");
    } else if (g.nq != want) {
        fail(QS_ERR_INVALID, "gate type " + std::to_string(g.type) + " takes " +
                                 std::to_string(want) + " qubits, got " + std::to_string(g.nq));
    }
    uint64_t seen = 0;
    for (int j = 0; j < g.nq; j++) {
        if (g.q[j] < 0 || g.q[j] >= n)
            fail(QS_ERR_INVALID, "qubit " + std::to_string(g.q[j]) + " out of range for " +
                                     std::to_string(n) + " qubits");
        if ((seen >> g.q[j]) & 1) fail(QS_ERR_INVALID, "repeated operand qubit");
        seen |= 1ull << g.q[j];
    }
    for (int j = 0; j < 3; j++)
        if (!std::isfinite(g.p[j])) fail(QS_ERR_INVALID, "non-finite gate parameter");
    if (g.type == QS_DENSE) {
        const size_t cnt = 2ull << (2 * g.nq);
        for (size_t i = 0; i < cnt; i++)
            if (!std::isfinite(g.m[i])) fail(QS_ERR_INVALID, "non-finite dense matrix entry");
    }
}

Op lower_gate(const qs_gate &g) {
    Op op;
    op.k = g.nq;
    for (int j = 0; j < g.nq; j++) op.q[j] = g.q[j];
    const double *p = g.p;
    switch (g.type) {
    case QS_H: op.kind = K_H; break;
    case QS_X: op.kind = K_PERM1; break;
    case QS_Y: op.kind = K_DENSE1; op.m = {0.0, -kI, kI, 0.0}; break;
    case QS_Z: op.kind = K_DIAG1; op.m = {1.0, -1.0}; break;
    case QS_S: op.kind = K_DIAG1; op.m = {1.0, kI}; break;
    case QS_T: op.kind = K_DIAG1; op.m = {1.0, std::polar(1.0, M_PI / 4)}; break;
    case QS_RX: {
        const double c = std::cos(0.5 * p[0]), s = std::sin(0.5 * p[0]);
        op.kind = K_DENSE1;
        op.m = {c, -kI * s, -kI * s, c};
        break;
    }
    case QS_RY: {
        const double c = std::cos(0.5 * p[0]), s = std::sin(0.5 * p[0]);
        op.kind = K_DENSE1;
        op.m = {c, -s, s, c};
        break;
    }
    case QS_RZ:
        op.kind = K_DIAG1;
        op.m = {std::polar(1.0, -0.5 * p[0]), std::polar(1.0, 0.5 * p[0])};
        break;
    case QS_P: op.kind = K_DIAG1; op.m = {1.0, std::polar(1.0, p[0])}; break;
    case QS_U3: op.kind = K_DENSE1; op.m = u3(p[0], p[1], p[2]); break;
    case QS_CNOT: op.kind = K_CTRL1; op.m = {0.0, 1.0, 1.0, 0.0}; break;
    case QS_CU3: op.kind = K_CTRL1; op.m = u3(p[0], p[1], p[2]); break;
    case QS_SWAP: op.kind = K_SWAP; break;
    case QS_CZ: op.kind = K_DIAG; op.m = {1.0, 1.0, 1.0, -1.0}; break;
    case QS_CP: op.kind = K_DIAG; op.m = {1.0, 1.0, 1.0, std::polar(1.0, p[0])}; break;
    case QS_RZZ: {
        const cd e = std::polar(1.0, -0.5 * p[0]), f = std::polar(1.0, 0.5 * p[0]);
        op.kind = K_DIAG;
        op.m = {e, f, f, e};
        break;
    }
    case QS_DENSE: {
        const size_t d = 1ull << g.nq;
        op.m.resize(d * d);
        for (size_t i = 0; i < d * d; i++) op.m[i] = cd(g.m[2 * i], g.m[2 * i + 1]);
        op.kind = g.nq == 1 ? K_DENSE1 : K_DENSE;
        break;
    }
    default:
        fail(QS_ERR_INVALID, "unknown gate type");
    }
    return op;
}

std::vector<cd> Op::full() const {
    const size_t d = 1ull << k;
    std::vector<cd> f(d * d, 0.0);
    switch (kind) {
    case K_H: {
        const double r = m.empty() ? 1.0 / std::sqrt(2.0) : m[0].real();
        f = {r, r, r, -r};
        break;
    }
    case K_PERM1: f = {0.0, 1.0, 1.0, 0.0}; break;
    case K_DIAG1: f = {m[0], 0.0, 0.0, m[1]}; break;
    case K_DENSE1: f = m; break;
    case K_CTRL1:   // rows/cols: (c,t) = 00, 01, 10, 11
        f[0] = 1.0;
        f[5] = 1.0;
        f[10] = m[0]; f[11] = m[1];
        f[14] = m[2]; f[15] = m[3];
        break;
    case K_SWAP: f[0] = 1.0; f[6] = 1.0; f[9] = 1.0; f[15] = 1.0; break;
    case K_DIAG:
        for (size_t i = 0; i < d; i++) f[i * d + i] = m[i];
        break;
    case K_DENSE: f = m; break;
    case K_PHASEFN: fail(QS_ERR_INVALID, "a phase function has no dense matrix");
    }
    return f;
}

namespace {

// Embeds op (on its own operand order) into the qubit list Q (Q[0] most significant):
// returns the 2^|Q| x 2^|Q| matrix acting as op on its qubits and as identity elsewhere.
std::vector<cd> embed(const Op &op, const std::vector<int> &Q) {
    const int K = (int)Q.size();
    const size_t D = 1ull << K;
    const std::vector<cd> f = op.full();
    const size_t d = 1ull << op.k;
    int pos[8];  // position (bit index within the Q sub-index) of each operand
    uint64_t opbits = 0;
    for (int j = 0; j < op.k; j++) {
        int found = -1;
        for (int t = 0; t < K; t++)
            if (Q[t] == op.q[j]) found = t;
        pos[j] = K - 1 - found;
        opbits |= 1ull << pos[j];
    }
    auto sub = [&](uint64_t r) {
        uint64_t s = 0;
        for (int j = 0; j < op.k; j++) s |= ((r >> pos[j]) & 1ull) << (op.k - 1 - j);
        return s;
    };
    std::vector<cd> out(D * D, 0.0);
    for (uint64_t r = 0; r < D; r++)
        for (uint64_t c = 0; c < D; c++) {
            if ((r & ~opbits) != (c & ~opbits)) continue;
            out[r * D + c] = f[sub(r) * d + sub(c)];
        }
    return out;
}

bool is_diagonal(const Op &op) { return op.kind == K_DIAG1 || op.kind == K_DIAG; }

}  // namespace

bool op_is_diagonal(const Op &op) {
    switch (op.kind) {
    case K_DIAG1: case K_DIAG: case K_PHASEFN: return true;
    case K_CTRL1: return op.m[1] == cd(0.0) && op.m[2] == cd(0.0);
    default: return false;
    }
}

std::vector<Op> fold_global_phases(const std::vector<Op> &ops) {
    std::vector<Op> out = ops;
    int last = -1;
    for (size_t i = 0; i < out.size(); i++)
        if (out[i].kind == K_DIAG1 && out[i].m[0] != cd(1.0)) last = (int)i;
    cd phase = 1.0;
    for (int i = 0; i < last; i++) {
        Op &op = out[i];
        if (op.kind != K_DIAG1 || op.m[0] == cd(1.0) || op.m[0] == cd(0.0)) continue;
        phase *= op.m[0];
        op.m = {cd(1.0), op.m[1] / op.m[0]};
    }
    if (last >= 0) out[last].m = {out[last].m[0] * phase, out[last].m[1] * phase};
    return out;
}

void defer_hadamard_scale(std::vector<Op> &ops) {
    int last = -1;
    for (size_t i = 0; i < ops.size(); i++)
        if (ops[i].kind == K_H) last = (int)i;
    int c = 0;  // unscaled Hadamards since the last scaled one
    for (int i = 0; i <= last; i++) {
        if (ops[i].kind != K_H) continue;
        if (i == last || c == kMaxUnscaledH) {
            const int k = c + 1;  // factor 2^(-k/2)
            const double r = (k % 2 == 0) ? std::ldexp(1.0, -k / 2) : std::ldexp(std::sqrt(0.5), -(k - 1) / 2);
            ops[i].m = {cd(r)};
            c = 0;
        } else {
            ops[i].m = {cd(1.0)};
            c++;
        }
    }
}

std::vector<Op> split_one_qubit_phases(const std::vector<Op> &ops) {
    // u = [[a, b], [c, d]] with real a: R = [[a, -s], [s, a]], s = |c|, e^{i phi} = c / s,
    // e^{i lambda} = -b / s; taken only where P(phi) R P(lambda) reproduces u, and only for
    // one-qubit matrices of the U3 class (real first entry, complex elsewhere: real and
    // RX-like matrices already cost 4; a controlled split costs two controlled phases).
    struct Parts {
        cd pl, pf;
        double a, s;
        bool diag;
    };
    auto split = [](const Op &op, Parts &r) {
        if (op.kind != K_DENSE1 || d1_class(op.m) != D1_R0) return false;
        const cd a = op.m[0], b = op.m[1], c = op.m[2], d = op.m[3];
        const double s = std::abs(c);
        if (s == 0.0) {  // already diagonal
            if (b != cd(0.0)) return false;
            r.diag = true;
            return true;
        }
        r.diag = false;
        r.a = a.real();
        r.s = s;
        r.pf = c / s;
        r.pl = -b / s;
        const double tol = 1e-14;
        if (std::abs(r.pl * (-s) - b) > tol || std::abs(r.pf * s - c) > tol ||
            std::abs(r.pf * r.pl * r.a - d) > tol)
            return false;
        return true;
    };
    auto part = [](const Op &src, std::vector<cd> u) {
        Op p;
        p.kind = src.kind;
        p.k = src.k;
        for (int j = 0; j < src.k; j++) p.q[j] = src.q[j];
        if (src.kind == K_DENSE1 && u[1] == cd(0.0) && u[2] == cd(0.0)) {
            p.kind = K_DIAG1;
            u = {u[0], u[3]};
        }
        p.m = std::move(u);
        return p;
    };
    std::vector<Op> out;
    size_t i = 0;
    while (i < ops.size()) {
        // a run of splittable ops on disjoint qubit sets
        size_t j = i;
        uint64_t seen = 0;
        std::vector<Parts> parts;
        while (j < ops.size()) {
            Parts pr;
            const uint64_t qm = ops[j].qmask();
            if ((qm & seen) || !split(ops[j], pr)) break;
            seen |= qm;
            parts.push_back(pr);
            j++;
        }
        if (j == i) {
            out.push_back(ops[i++]);
            continue;
        }
        for (size_t t = i; t < j; t++) {  // P(lambda) of every member, then R, then P(phi)
            const Parts &pr = parts[t - i];
            out.push_back(part(ops[t], pr.diag ? ops[t].m : std::vector<cd>{cd(1.0), cd(0.0), cd(0.0), pr.pl}));
        }
        for (size_t t = i; t < j; t++) {
            const Parts &pr = parts[t - i];
            if (!pr.diag) out.push_back(part(ops[t], {cd(pr.a), cd(-pr.s), cd(pr.s), cd(pr.a)}));
        }
        for (size_t t = i; t < j; t++) {
            const Parts &pr = parts[t - i];
            if (!pr.diag) out.push_back(part(ops[t], {cd(1.0), cd(0.0), cd(0.0), pr.pf}));
        }
        i = j;
    }
    return out;
}

double op_flops(const Op &op) {
    // FP64 operations per amplitude of the one-qubit forms (general 8, real first entry 7,
    // real 4, RX-like 4)
    auto dense1 = [](const std::vector<cd> &u) {
        switch (d1_class(u)) {
        case D1_REAL: case D1_RX: return 4.0;
        case D1_R0: return 7.0;
        default: return 8.0;
        }
    };
    switch (op.kind) {
    case K_H: return (!op.m.empty() && op.m[0] == cd(1.0)) ? 2.0 : 3.0;
    case K_PERM1: case K_SWAP: return 0.0;
    case K_DIAG1: return op.m[0] == cd(1.0) ? 2.0 : 4.0;
    case K_DENSE1: return dense1(op.m);
    case K_CTRL1: return 0.5 * dense1(op.m);
    case K_DIAG: return 4.0;
    case K_DENSE: return 4.0 * (double)(1 << op.k);
    case K_PHASEFN: return 6.0;
    }
    return 8.0;
}

namespace {

// Diagonal entries of op on its own operands (first operand most significant), if it is
// a diagonal (K_DIAG1, K_DIAG, or K_CTRL1 with a diagonal 2x2).
bool diag_of(const Op &op, std::vector<cd> &d) {
    switch (op.kind) {
    case K_DIAG1:
    case K_DIAG:
        d = op.m;
        return true;
    case K_CTRL1:
        if (op.m[1] != cd(0.0) || op.m[2] != cd(0.0)) return false;
        d = {1.0, 1.0, op.m[0], op.m[3]};
        return true;
    default:
        return false;
    }
}

// FP64 operations per amplitude of one diagonal applied alone in a shared-memory sweep of
// a complex128 tile: a complex multiply is 4, restricted to the fraction of elements it
// changes; a sign flip is free.
double diag_cost(const std::vector<cd> &d) {
    size_t changed = 0;
    bool neg_only = true;
    for (const cd &z : d)
        if (z != cd(1.0)) {
            changed++;
            neg_only = neg_only && z == cd(-1.0);
        }
    if (changed == 0 || neg_only) return 0.0;
    // the kernels restrict work to the elements with the controls set (phase on |1..1>)
    if (changed == 1 && d.back() != cd(1.0)) return 4.0 / (double)d.size();
    return 4.0;
}

}  // namespace

uint64_t hi_local_choices(const Op &op) {
    std::vector<cd> d;
    if (!(op.kind == K_CTRL1 || (op.kind == K_DIAG && op.k == 2)) || !diag_of(op, d)) return 0;
    for (const cd &z : d)
        if (z == cd(0.0)) return 0;
    // d over (q0, q1), q0 most significant: q0 may stay local if d(0, x) = 1, q1 if d(x, 0) = 1
    uint64_t r = 0;
    if (d[0] == cd(1.0) && d[1] == cd(1.0)) r |= 1ull << op.q[0];
    if (d[0] == cd(1.0) && d[2] == cd(1.0)) r |= 1ull << op.q[1];
    return r;
}

std::vector<Op> merge_tile_diagonals(std::vector<Op> ops, int max_k, double sweep_cost, uint64_t lmask) {
    std::vector<Op> out;
    std::vector<int> Q;                  // block qubits (local), Q[0] most significant
    std::vector<cd> D;                   // block diagonal over Q
    std::vector<HiTerm> terms;           // factors from non-local qubits
    std::vector<Op *> members;           // ops of the open block (moved out when it is split)
    bool forced = false;                 // a member has a non-local qubit: emit the block
    double member_cost = 0.0;
    auto is_local = [&](int q) { return lmask == 0 || ((lmask >> q) & 1ull) != 0; };
    // controls: qubits on whose 0-half every entry is 1 and to which every HiTerm is tied;
    // a block costs a complex multiply on the elements with all controls set, and its
    // table covers the other qubits only
    auto controls = [](const std::vector<int> &q, const std::vector<cd> &d, const std::vector<HiTerm> &tt) {
        const int K = (int)q.size();
        int nctl = 0;
        for (int j = 0; j < K; j++) {
            const int bit = K - 1 - j;
            bool ctl = true;
            for (size_t x = 0; x < d.size() && ctl; x++)
                if (!((x >> bit) & 1) && d[x] != cd(1.0)) ctl = false;
            for (const HiTerm &t : tt) ctl = ctl && t.t == q[j];
            nctl += ctl;
        }
        return nctl;
    };
    auto flush = [&]() {
        if (members.empty()) return;
        const int K = (int)Q.size();
        const int nctl = controls(Q, D, terms);
        bool identity = terms.empty();
        for (const cd &z : D) identity = identity && z == cd(1.0);
        const double merged = identity ? 0.0 : 4.0 / (double)(1u << nctl) + sweep_cost;
        if (forced || (members.size() >= 2 && merged < member_cost)) {
            if (!identity) {
                Op b;
                b.kind = K_DIAG;
                b.k = K;
                for (int j = 0; j < K; j++) b.q[j] = Q[j];
                b.m = D;
                b.hi = terms;
                out.push_back(std::move(b));
            }
        } else {
            for (Op *m : members) out.push_back(std::move(*m));
        }
        members.clear();
        Q.clear();
        D.clear();
        terms.clear();
        forced = false;
        member_cost = 0.0;
    };
    // per-op scratch, reused across ops (the block's vectors trade buffers with it)
    std::vector<cd> d, dl, nD;
    std::vector<int> lq, nQ;
    std::vector<HiTerm> nt, nterms;
    for (Op &op : ops) {
        if (!diag_of(op, d)) {
            flush();
            out.push_back(std::move(op));
            continue;
        }
        // the op's local part: its diagonal on its local qubits, with the x_h = 0 slice
        // and HiTerms for a non-local qubit h (two-qubit diagonals only)
        int jh = -1;
        for (int j = 0; j < op.k; j++)
            if (!is_local(op.q[j])) jh = j;
        nt.clear();
        if (jh < 0) {
            lq.assign(op.q, op.q + op.k);
            dl = d;
        } else {
            if (op.k != 2 || !((hi_local_choices(op) >> op.q[1 - jh]) & 1ull))
                fail(QS_ERR_INVALID, "internal: diagonal with a non-local qubit");
            const int ja = 1 - jh, qa = op.q[ja], qh = op.q[jh];
            auto dd = [&](int xa, int xh) {
                return d[(size_t)(((ja == 0 ? xa : xh) << 1) | (ja == 0 ? xh : xa))];
            };
            lq = {qa};
            dl = {dd(0, 0), dd(1, 0)};
            const cd g0 = dd(0, 1) / dd(0, 0), g1 = dd(1, 1) / dd(1, 0);
            if (g0 != cd(1.0)) nt.push_back({-1, qh, g0});
            const cd r = g1 / g0;
            if (r != cd(1.0)) nt.push_back({qa, qh, r});
        }
        // the block with this op: qubits high-to-low, entries, terms
        auto extend = [&](std::vector<int> &nQ, std::vector<cd> &nD, std::vector<HiTerm> &nterms) {
            const bool fresh = members.empty();
            nQ = fresh ? lq : Q;
            if (!fresh)
                for (int q : lq)
                    if (std::find(nQ.begin(), nQ.end(), q) == nQ.end()) nQ.push_back(q);
            std::sort(nQ.begin(), nQ.end(), [](int a, int b) { return a > b; });
            const int K = (int)nQ.size();
            const int kl = (int)lq.size();
            nD.assign((size_t)1 << K, 1.0);
            for (size_t x = 0; x < nD.size(); x++) {
                auto bit_of = [&](int q) {
                    for (int t = 0; t < K; t++)
                        if (nQ[t] == q) return (int)((x >> (K - 1 - t)) & 1);
                    return 0;
                };
                size_t xo = 0;  // index into the old block
                for (size_t t = 0; t < Q.size(); t++) xo |= (size_t)bit_of(Q[t]) << (Q.size() - 1 - t);
                size_t xm = 0;  // index into the op's local diagonal
                for (int j = 0; j < kl; j++) xm |= (size_t)bit_of(lq[j]) << (kl - 1 - j);
                nD[x] = (fresh ? cd(1.0) : D[xo]) * dl[xm];
            }
            nterms = fresh ? nt : terms;
            if (!fresh) nterms.insert(nterms.end(), nt.begin(), nt.end());
        };
        // limits: at most max_k qubits; a table of at most 2^max_k entries, 2^(max_k - 1)
        // with terms (so that table and terms fit one op's reals, and every table bit
        // with terms has a factor slot)
        auto fits = [&](const std::vector<int> &q, const std::vector<cd> &d, const std::vector<HiTerm> &tt) {
            const int table_bits = (int)q.size() - controls(q, d, tt);
            return (int)q.size() <= max_k && table_bits <= (tt.empty() ? max_k : max_k - 1) &&
                   tt.size() <= (size_t)kMaxHiTerms;
        };
        extend(nQ, nD, nterms);
        if (!members.empty() && !fits(nQ, nD, nterms)) {
            flush();
            extend(nQ, nD, nterms);
        }
        Q.swap(nQ);
        D.swap(nD);
        terms.swap(nterms);
        members.push_back(&op);
        forced = forced || jh >= 0;
        member_cost += diag_cost(d) + sweep_cost;
    }
    flush();
    return out;
}

std::vector<Op> fuse_ops(std::vector<Op> ops, int fuse_k, double sweep_flops, uint64_t lmask) {
    if (fuse_k <= 1) return ops;
    std::vector<Op> out;
    std::vector<int> Q;                  // qubits of the current block, Q[0] most significant
    std::vector<cd> U;                   // its matrix
    std::vector<Op *> members;           // ops absorbed into the current block
    bool diag = true;
    double member_flops = 0.0;           // flops/amplitude of the members applied one by one
    std::vector<int> nQ;                 // scratch: qubits of the block with the next op

    auto flush = [&]() {
        if (members.empty()) return;
        if (members.size() == 1) {
            out.push_back(std::move(*members[0]));
        } else {
            Op b;
            b.k = (int)Q.size();
            for (int j = 0; j < b.k; j++) b.q[j] = Q[j];
            const size_t D = 1ull << b.k;
            if (diag) {
                b.kind = b.k == 1 ? K_DIAG1 : K_DIAG;
                b.m.resize(D);
                for (size_t i = 0; i < D; i++) b.m[i] = U[i * D + i];
            } else {
                b.kind = b.k == 1 ? K_DENSE1 : K_DENSE;
                b.m = U;
            }
            out.push_back(std::move(b));
        }
        members.clear();
        Q.clear();
        U.clear();
        diag = true;
        member_flops = 0.0;
    };

    for (Op &op : ops) {
        if (lmask && (op.qmask() & ~lmask)) {
            // a gate with a qubit outside the pass's local set is applied on its own
            flush();
            out.push_back(std::move(op));
            continue;
        }
        const double f_op = op_flops(op);
        const bool op_diag = is_diagonal(op);
        nQ.assign(Q.begin(), Q.end());
        for (int j = 0; j < op.k; j++) {
            bool have = false;
            for (int x : nQ) have |= x == op.q[j];
            if (!have) nQ.push_back(op.q[j]);
        }
        bool fits = (int)nQ.size() <= fuse_k;
        if (fits && !members.empty() && sweep_flops >= 0.0) {
            // cost gate: the fused block may not cost more flops per amplitude than its
            // members one by one plus the saved shared-memory sweep
            const bool ndiag = diag && op_diag;
            const double fused = ndiag ? 4.0 : 4.0 * (double)(1 << nQ.size());
            fits = fused <= member_flops + f_op + sweep_flops;
        }
        if (!fits) {
            flush();
            nQ.assign(op.q, op.q + op.k);
        }
        // keep the block's qubits sorted high-to-low so that equal sets give equal orders
        std::sort(nQ.begin(), nQ.end(), [](int a, int b) { return a > b; });
        const size_t D = 1ull << nQ.size();
        // a block of one op is emitted as that op: its matrix is formed when a second joins
        std::vector<cd> newU;
        if (!members.empty()) {
            std::vector<cd> A;
            if (members.size() == 1) {
                A = embed(*members[0], nQ);
            } else {
                Op cur;
                cur.kind = K_DENSE;
                cur.k = (int)Q.size();
                for (int j = 0; j < cur.k; j++) cur.q[j] = Q[j];
                cur.m = U;
                A = embed(cur, nQ);
            }
            const std::vector<cd> B = embed(op, nQ);
            newU.assign(D * D, 0.0);
            for (size_t r = 0; r < D; r++)
                for (size_t t = 0; t < D; t++) {
                    const cd b = B[r * D + t];
                    if (b == cd(0.0)) continue;
                    for (size_t c = 0; c < D; c++) newU[r * D + c] += b * A[t * D + c];
                }
        }
        Q.assign(nQ.begin(), nQ.end());
        U = std::move(newU);
        members.push_back(&op);
        member_flops += f_op;
        diag = diag && op_diag;
    }
    flush();
    return out;
}

}  // namespace qs
