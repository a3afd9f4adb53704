// Host: lowered Op -> kernel-side KOp in a given index space, plus algorithmic bytes.
#include <algorithm>
#include <cmath>

#include "kgeom.h"

namespace qs {

int32_t d1_class(const std::vector<cd> &u) {
    const bool real = u[0].imag() == 0.0 && u[1].imag() == 0.0 && u[2].imag() == 0.0 && u[3].imag() == 0.0;
    if (real) return D1_REAL;
    if (u[0].imag() == 0.0 && u[3].imag() == 0.0 && u[1].real() == 0.0 && u[2].real() == 0.0) return D1_RX;
    if (u[0].imag() == 0.0) return D1_R0;
    return D1_GENERAL;
}

namespace {

bool is_one(cd z) { return z == cd(1.0, 0.0); }

bool is_minus_one(cd z) { return z == cd(-1.0, 0.0); }

void push_c(std::vector<double> &mats, KOp &k, std::initializer_list<cd> vals) {
    k.mat = (int32_t)mats.size();
    for (cd v : vals) {
        mats.push_back(v.real());
        mats.push_back(v.imag());
    }
    k.nmat = (int32_t)mats.size() - k.mat;
}

void push_vec(std::vector<double> &mats, KOp &k, const std::vector<cd> &vals) {
    k.mat = (int32_t)mats.size();
    for (cd v : vals) {
        mats.push_back(v.real());
        mats.push_back(v.imag());
    }
    k.nmat = (int32_t)mats.size() - k.mat;
}

KOp base(int fkind, std::initializer_list<int> fixed, uint64_t set_mask,
         std::initializer_list<uint64_t> offs) {
    KOp k{};
    k.fkind = fkind;
    k.nf = 0;
    for (int b : fixed) k.fb[k.nf++] = b;
    std::sort(k.fb, k.fb + k.nf);
    k.set_mask = set_mask;
    k.nt = 0;
    for (uint64_t o : offs) k.off[k.nt++] = o;
    k.mat = k.nmat = 0;
    return k;
}

// phase/neg on the single element with every bit of `bits` set
KOp phase_on(std::initializer_list<int> bits, cd ph, std::vector<double> &mats) {
    uint64_t set = 0;
    for (int b : bits) set |= 1ull << b;
    KOp k = base(is_minus_one(ph) ? F_NEG : F_PHASE, bits, set, {0});
    if (k.fkind == F_PHASE) push_c(mats, k, {ph});
    return k;
}

}  // namespace

KOp make_kop(const Op &op, const int *pos, std::vector<double> &mats) {
    auto P = [&](int j) { return pos[op.q[j]]; };
    switch (op.kind) {
    case K_H: {
        const int p = P(0);
        KOp k = base(F_H, {p}, 0, {0, 1ull << p});
        if (!op.m.empty()) push_c(mats, k, {op.m[0]});  // scale (re, 0) instead of 1/sqrt2
        return k;
    }
    case K_PERM1: {
        const int p = P(0);
        return base(F_SWAP, {p}, 0, {0, 1ull << p});
    }
    case K_DIAG1: {
        const int p = P(0);
        if (is_one(op.m[0])) return phase_on({p}, op.m[1], mats);
        KOp k = base(F_DIAG1, {p}, 0, {0, 1ull << p});
        push_c(mats, k, {op.m[0], op.m[1]});
        return k;
    }
    case K_DENSE1: {
        const int p = P(0);
        KOp k = base(F_DENSE1, {p}, 0, {0, 1ull << p});
        k.k = d1_class(op.m);
        push_vec(mats, k, op.m);
        return k;
    }
    case K_CTRL1: {
        const int c = P(0), t = P(1);
        const std::vector<cd> &u = op.m;
        const bool diag = u[1] == cd(0.0) && u[2] == cd(0.0);
        if (u[0] == cd(0.0) && u[3] == cd(0.0) && is_one(u[1]) && is_one(u[2]))
            return base(F_SWAP, {c, t}, 1ull << c, {0, 1ull << t});
        if (diag && is_one(u[0])) return phase_on({c, t}, u[3], mats);
        if (diag) {
            KOp k = base(F_DIAG1, {c, t}, 1ull << c, {0, 1ull << t});
            push_c(mats, k, {u[0], u[3]});
            return k;
        }
        KOp k = base(F_DENSE1, {c, t}, 1ull << c, {0, 1ull << t});
        k.k = d1_class(u);
        push_vec(mats, k, u);
        return k;
    }
    case K_SWAP: {
        const int a = P(0), b = P(1);
        return base(F_SWAP, {a, b}, 0, {1ull << a, 1ull << b});
    }
    case K_DIAG: {
        if (op.k == 1) {
            const int p = P(0);
            if (is_one(op.m[0])) return phase_on({p}, op.m[1], mats);
            KOp k = base(F_DIAG1, {p}, 0, {0, 1ull << p});
            push_c(mats, k, {op.m[0], op.m[1]});
            return k;
        }
        if (op.k == 2) {
            const int a = P(0), b = P(1);
            if (is_one(op.m[0]) && is_one(op.m[1]) && is_one(op.m[2])) return phase_on({a, b}, op.m[3], mats);
            const uint64_t A = 1ull << a, B = 1ull << b;
            KOp k = base(F_DIAG2, {a, b}, 0, {0, B, A, A | B});
            push_vec(mats, k, op.m);
            return k;
        }
        KOp k{};
        k.fkind = F_DIAGK;
        k.k = op.k;
        for (int j = 0; j < op.k; j++) k.pos[j] = P(j);
        push_vec(mats, k, op.m);
        return k;
    }
    case K_DENSE: {
        if (op.k == 2) {
            const int a = P(0), b = P(1);
            const uint64_t A = 1ull << a, B = 1ull << b;
            KOp k = base(F_DENSE2, {a, b}, 0, {0, B, A, A | B});
            push_vec(mats, k, op.m);
            return k;
        }
        KOp k{};
        k.fkind = F_DENSEK;
        k.k = op.k;
        for (int j = 0; j < op.k; j++) k.pos[j] = P(j);
        push_vec(mats, k, op.m);
        return k;
    }
    }
    fail(QS_ERR_INVALID, "unknown op kind");
}

namespace {

// A diagonal block with factors from non-local qubits: F_CDIAGK whose reals hold the table
// over its non-control positions, then nt terms (table bit or -1, global qubit, re, im).
// Controls: qubits on whose 0-half the table is 1 and to which every term is tied (every
// visited element has them set, so such a term applies to the whole table).
KOp make_hi_block_kop(const Op &op, const int *pos, std::vector<double> &mats) {
    const int K = op.k;
    std::vector<int> ctl, tab;  // operand indices
    for (int j = 0; j < K; j++) {
        const int bit = K - 1 - j;
        bool c = true;
        for (size_t x = 0; x < op.m.size() && c; x++)
            if (!((x >> bit) & 1) && op.m[x] != cd(1.0)) c = false;
        for (const HiTerm &t : op.hi) c = c && t.t == op.q[j];
        (c ? ctl : tab).push_back(j);
    }
    KOp k{};
    k.fkind = F_CDIAGK;
    k.k = (int)tab.size();
    for (int i = 0; i < k.k; i++) k.pos[i] = pos[op.q[tab[i]]];
    std::vector<int> cp;
    for (int j : ctl) cp.push_back(pos[op.q[j]]);
    std::sort(cp.begin(), cp.end());
    k.nf = (int)cp.size();
    for (int i = 0; i < k.nf; i++) {
        k.pos[k.k + i] = cp[i];
        k.set_mask |= 1ull << cp[i];
    }
    k.mat = (int32_t)mats.size();
    for (size_t s = 0; s < (1ull << k.k); s++) {
        size_t x = 0;
        for (int j : ctl) x |= (size_t)1 << (K - 1 - j);
        for (int i = 0; i < k.k; i++)
            if ((s >> (k.k - 1 - i)) & 1) x |= (size_t)1 << (K - 1 - tab[i]);
        mats.push_back(op.m[x].real());
        mats.push_back(op.m[x].imag());
    }
    for (const HiTerm &t : op.hi) {
        int tb = -1;
        for (int i = 0; i < k.k; i++)
            if (op.q[tab[i]] == t.t) tb = k.k - 1 - i;
        k.off[0] |= 1ull << (tb + 1);  // which factors the kernel has to build
        mats.push_back((double)tb);
        mats.push_back((double)t.h);
        mats.push_back(t.f.real());
        mats.push_back(t.f.imag());
    }
    k.nt = (int32_t)op.hi.size();
    k.nmat = (int32_t)mats.size() - k.mat;
    if (k.nmat > kMaxOpReals) fail(QS_ERR_INVALID, "internal: diagonal block too large");
    return k;
}

}  // namespace

KOp make_tile_kop(const Op &op, const int *pos, std::vector<double> &mats) {
    if (op.kind == K_DIAG && !op.hi.empty()) return make_hi_block_kop(op, pos, mats);
    if (op.kind != K_DIAG || op.k < 3) return make_kop(op, pos, mats);
    const int K = op.k;
    std::vector<int> ctl, tab;  // operand indices
    for (int j = 0; j < K; j++) {
        const int bit = K - 1 - j;
        bool c = true;
        for (size_t x = 0; x < op.m.size() && c; x++)
            if (!((x >> bit) & 1) && op.m[x] != cd(1.0)) c = false;
        (c ? ctl : tab).push_back(j);
    }
    if (ctl.empty()) return make_kop(op, pos, mats);
    KOp k{};
    k.fkind = F_CDIAGK;
    k.k = (int)tab.size();
    for (int i = 0; i < k.k; i++) k.pos[i] = pos[op.q[tab[i]]];
    std::vector<int> cp;
    for (int j : ctl) cp.push_back(pos[op.q[j]]);
    std::sort(cp.begin(), cp.end());
    k.nf = (int)cp.size();
    for (int i = 0; i < k.nf; i++) {
        k.pos[k.k + i] = cp[i];
        k.set_mask |= 1ull << cp[i];
    }
    k.mat = (int32_t)mats.size();
    for (size_t s = 0; s < (1ull << k.k); s++) {
        size_t x = 0;  // operand index with every control set and the table bits from s
        for (int j : ctl) x |= (size_t)1 << (K - 1 - j);
        for (int i = 0; i < k.k; i++)
            if ((s >> (k.k - 1 - i)) & 1) x |= (size_t)1 << (K - 1 - tab[i]);
        mats.push_back(op.m[x].real());
        mats.push_back(op.m[x].imag());
    }
    k.nmat = (int32_t)mats.size() - k.mat;
    return k;
}

std::vector<KOp> join_h_cdiag(const std::vector<KOp> &kops, const std::vector<double> &mats) {
    std::vector<KOp> out;
    out.reserve(kops.size());
    for (size_t i = 0; i < kops.size(); i++) {
        const KOp &h = kops[i];
        const bool unscaled_h = h.fkind == F_H && h.nmat == 2 && mats[(size_t)h.mat] == 1.0 &&
                                mats[(size_t)h.mat + 1] == 0.0;
        if (unscaled_h && i + 1 < kops.size()) {
            const KOp &d = kops[i + 1];
            if (d.fkind == F_CDIAGK && d.nf == 1 && d.pos[d.k] == h.fb[0]) {
                KOp j = d;
                j.fkind = F_HCDIAGK;
                out.push_back(j);
                i++;
                continue;
            }
        }
        out.push_back(h);
    }
    return out;
}

namespace {

// One op as a register-phase member (tile positions); false if a phase cannot hold it.
struct RpMember {
    int type = 0;
    int tgt = -1;       // register-slot operand (a position the phase must hold in registers)
    int a = -1, b = -1; // position operands (-1: bit 1 for every amplitude, -2: bit 0)
    int form = RP_GENERAL;  // RP_M1: RP_GENERAL / RP_REAL / RP_RX
    double pay[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

bool rp_member(const Op &op, const int *pos, RpMember &mb) {
    auto P = [&](int j) { return pos[op.q[j]]; };
    auto put = [&](int i, cd z) {
        mb.pay[2 * i] = z.real();
        mb.pay[2 * i + 1] = z.imag();
    };
    auto mat = [&](cd m00, cd m01, cd m10, cd m11) {
        put(0, m00); put(1, m01); put(2, m10); put(3, m11);
    };
    // a one-qubit M1 in its cheapest form
    auto m1 = [&](cd m00, cd m01, cd m10, cd m11) {
        mb.type = RP_M1;
        if (m00.imag() == 0.0 && m01.imag() == 0.0 && m10.imag() == 0.0 && m11.imag() == 0.0) {
            mb.form = RP_REAL;
            mb.pay[0] = m00.real(); mb.pay[1] = m01.real(); mb.pay[2] = m10.real(); mb.pay[3] = m11.real();
        } else if (m00.imag() == 0.0 && m11.imag() == 0.0 && m01.real() == 0.0 && m10.real() == 0.0) {
            mb.form = RP_RX;
            mb.pay[0] = m00.real(); mb.pay[1] = m01.imag(); mb.pay[2] = m10.imag(); mb.pay[3] = m11.real();
        } else {
            mb.form = RP_GENERAL;
            mat(m00, m01, m10, m11);
        }
    };
    // diagonal on positions (a, b), entry index 2 x_a + x_b
    auto diag = [&](int a, int b, cd d0, cd d1, cd d2, cd d3) {
        mb.a = a;
        mb.b = b;
        if (is_one(d0) && is_one(d1) && is_one(d2)) {
            if (is_minus_one(d3)) {
                mb.type = RP_NEG;
            } else {
                mb.type = RP_PH;
                put(0, d3);
            }
        } else if (d0 == d3 && d1 == d2) {
            mb.type = RP_PARITY;  // depends on x_a xor x_b only (RZZ)
            put(0, d0); put(1, d1);
        } else {
            mb.type = RP_DIAG;
            put(0, d0); put(1, d1); put(2, d2); put(3, d3);
        }
    };
    // diagonal diag(d0, d1) on one position a
    auto diag1 = [&](int a, cd d0, cd d1) {
        mb.a = a;
        mb.b = a;
        if (is_one(d0) && is_minus_one(d1)) {
            mb.type = RP_NEG;
        } else if (is_one(d0)) {
            mb.type = RP_PH;
            put(0, d1);
        } else {
            mb.type = RP_PARITY;  // x_a xor 0 = x_a
            mb.b = -2;
            put(0, d0); put(1, d1);
        }
    };
    switch (op.kind) {
    case K_H: {
        const double r = 1.0 / std::sqrt(2.0);
        mb.tgt = P(0);
        m1(r, r, r, -r);
        return true;
    }
    case K_PERM1:
        mb.type = RP_X;
        mb.tgt = P(0);
        return true;
    case K_DENSE1:
        mb.tgt = P(0);
        m1(op.m[0], op.m[1], op.m[2], op.m[3]);
        return true;
    case K_DIAG1:
        diag1(P(0), op.m[0], op.m[1]);
        return true;
    case K_CTRL1: {
        const std::vector<cd> &u = op.m;
        if (u[1] == cd(0.0) && u[2] == cd(0.0)) {
            diag(P(0), P(1), 1.0, 1.0, u[0], u[3]);
            return true;
        }
        mb.tgt = P(1);
        mb.a = P(0);
        if (u[0] == cd(0.0) && u[3] == cd(0.0) && is_one(u[1]) && is_one(u[2])) {
            mb.type = RP_X;
        } else {
            mb.type = RP_C1;
            mat(u[0], u[1], u[2], u[3]);
        }
        return true;
    }
    case K_DIAG:
        if (op.k == 1) {
            diag1(P(0), op.m[0], op.m[1]);
            return true;
        }
        if (op.k == 2) {
            diag(P(0), P(1), op.m[0], op.m[1], op.m[2], op.m[3]);
            return true;
        }
        return false;
    default:
        return false;
    }
}

uint32_t tile_mask(const Op &op, const int *pos) {
    uint32_t r = 0;
    for (int j = 0; j < op.k; j++) r |= 1u << pos[op.q[j]];
    return r;
}

}  // namespace

bool rphase_applicable(int m, int thread_bits) { return m - thread_bits == kRpBits; }

std::vector<KOp> build_register_phases(const std::vector<Op> &ops, const int *pos, int m, int thread_bits,
                                       std::vector<double> &mats, int *n_phases) {
    if (!rphase_applicable(m, thread_bits)) fail(QS_ERR_INVALID, "register phases need m = thread bits + 5");
    const size_t N = ops.size();
    std::vector<RpMember> mb(N);
    std::vector<char> ok(N), done(N, 0);
    std::vector<uint32_t> touch(N);
    for (size_t i = 0; i < N; i++) {
        ok[i] = rp_member(ops[i], pos, mb[i]);
        touch[i] = tile_mask(ops[i], pos);
    }
    const uint32_t all = (1u << m) - 1u;
    // One greedy phase from `first`: an op joins if none of its positions is blocked by an
    // earlier op left out, its register operand fits in R (at most kRpBits positions,
    // within `allowed`) and the program has room; otherwise its positions become blocked.
    // diagonal ops commute with one another: one left out only blocks later non-diagonal ops
    std::vector<char> diag(N);
    for (size_t i = 0; i < N; i++) diag[i] = op_is_diagonal(ops[i]);
    auto trial = [&](size_t first, uint32_t allowed, std::vector<int> &taken) {
        uint32_t R = 0, blocked = 0, blocked_diag = 0;
        taken.clear();
        for (size_t i = first; i < N; i++) {
            if (done[i]) continue;
            const uint32_t tm = touch[i];
            const uint32_t blk = diag[i] ? blocked : (blocked | blocked_diag);
            bool take = ok[i] && !(tm & blk) && (int)taken.size() < kRpMaxMembers;
            if (take && mb[i].tgt >= 0) {
                const uint32_t need = 1u << mb[i].tgt;
                take = (need & ~allowed) == 0 && __builtin_popcount(R | need) <= kRpBits;
                if (take) R |= need;
            }
            if (take) taken.push_back((int)i);
            else if (diag[i]) blocked_diag |= tm;
            else blocked |= tm;
            if ((blocked & all) == all) break;
        }
        return R;
    };
    std::vector<KOp> out;
    int phases = 0;
    size_t first = 0;
    std::vector<int> best, cand;
    while (true) {
        while (first < N && done[first]) first++;
        if (first >= N) break;
        if (!ok[first]) {
            out.push_back(make_tile_kop(ops[first], pos, mats));
            done[first] = 1;
            continue;
        }
        // candidates: unrestricted, and register positions within each window of kRpBits
        // consecutive positions; keep the one that takes most ops
        uint32_t R = trial(first, all, best);
        for (int w = 0; w + kRpBits <= m; w++) {
            const uint32_t Rw = trial(first, ((1u << kRpBits) - 1u) << w, cand);
            if (cand.size() > best.size()) {
                best.swap(cand);
                R = Rw;
            }
        }
        // pad R with the highest free positions
        for (int p = m - 1; p >= 0 && __builtin_popcount(R) < kRpBits; p--) R |= 1u << p;
        KOp k{};
        k.fkind = F_RPHASE;
        k.k = kRpBits;
        int slot_of[32], tbit_of[32];
        int ns = 0, nt = 0;
        uint64_t tpos = 0;
        for (int p = 0; p < m; p++) {
            if ((R >> p) & 1u) {
                k.pos[ns] = p;
                slot_of[p] = ns++;
            } else {
                tpos |= (uint64_t)p << (4 * nt);
                tbit_of[p] = nt++;
            }
        }
        k.nt = nt;
        k.off[0] = tpos;
        auto enc = [&](int p) {
            if (p == -1) return kRpAlways;
            if (p == -2) return kRpNever;
            return ((R >> p) & 1u) ? 16 + slot_of[p] : tbit_of[p];
        };
        // members in order; consecutive sign flips merge (their patterns XOR), consecutive
        // parity diagonals with equal factors merge (a count of odd patterns, one table)
        struct Pending {
            int type, slot, ea, eb;
            std::vector<double> pay;
            std::vector<int> pairs;
            cd e, f;
        };
        // consecutive one-position phases and sign pairs (diagonal, so in any order) collect in
        // a run that becomes one RP_PH member in its run form (slot field 1) when it holds
        // at least kRpMinRunPhases phases; pay: (position, re, im) per phase
        constexpr int kPhaseRun = -1;
        std::vector<Pending> pend;
        uint32_t x_slots = 0;  // slots an exchange may have relabelled (bits of sigma it toggles)
        for (int i : best) {
            const RpMember &e = mb[i];
            done[i] = 1;
            if (e.type == RP_X) x_slots |= 1u << slot_of[e.tgt];
            const int ea = enc(e.a), eb = enc(e.b), pair = ea | eb << 5;
            Pending *last = pend.empty() ? nullptr : &pend.back();
            const bool one_pos_phase = e.type == RP_PH && e.a == e.b;
            if (one_pos_phase || e.type == RP_NEG) {
                if (!last || last->type != kPhaseRun || (int)last->pay.size() / 3 >= kRpMaxRunPhases ||
                    (int)last->pairs.size() >= kRpMaxRunPairs)
                    pend.push_back({kPhaseRun, 0, 0, 0, {}, {}, 0.0, 0.0});
                Pending &run = pend.back();
                if (one_pos_phase) {
                    run.pay.push_back((double)ea);
                    run.pay.push_back(e.pay[0]);
                    run.pay.push_back(e.pay[1]);
                } else {
                    run.pairs.push_back(pair);
                }
                continue;
            }
            if (e.type == RP_PARITY) {
                const cd ev(e.pay[0], e.pay[1]), fv(e.pay[2], e.pay[3]);
                if (last && last->type == RP_PARITY && last->e == ev && last->f == fv &&
                    (int)last->pairs.size() < kRpMaxParity)
                    last->pairs.push_back(pair);
                else pend.push_back({RP_PARITY, 0, 0, 0, {}, {pair}, ev, fv});
                continue;
            }
            // a 2x2 member carries its form in operand b
            Pending p{e.type, e.tgt >= 0 ? slot_of[e.tgt] : 0, ea, e.type == RP_M1 ? e.form : eb, {}, {}, 0.0, 0.0};
            const int npay = e.type == RP_X ? 0 : e.type == RP_PH ? 2
                             : (e.type == RP_M1 && e.form != RP_GENERAL) ? 4 : 8;
            p.pay.assign(e.pay, e.pay + npay);
            // a general matrix with a real first entry on a slot that no lane conjugates
            // (positions 4 and up carry no bit of sigma at the phase's start, and no
            // exchange on the slot has toggled it since): 7 multiply-adds instead of 8
            if (e.type == RP_M1 && e.form == RP_GENERAL && e.pay[1] == 0.0 && e.tgt >= 4 &&
                !((x_slots >> slot_of[e.tgt]) & 1u)) {
                p.eb = RP_R0;
                p.pay = {e.pay[0], e.pay[2], e.pay[3], e.pay[4], e.pay[5], e.pay[6], e.pay[7]};
            }
            pend.push_back(std::move(p));
        }
        k.mat = (int32_t)mats.size();
        mats.push_back(0.0);  // member count, set below (a short run of phases emits several)
        int n_emitted = 0;
        auto emit = [&](int type, int slot, int ea, int eb, const std::vector<double> &pay) {
            n_emitted++;
            // the device reads codes below 2^23 without a conversion instruction
            if (pay.size() >= 128) fail(QS_ERR_INVALID, "internal: register-phase member payload too long");
            mats.push_back((double)(type | slot << 3 | ea << 6 | eb << 11 | (int)pay.size() << 16));
            mats.insert(mats.end(), pay.begin(), pay.end());
        };
        for (const Pending &p : pend) {
            if (p.type == kPhaseRun) {
                const int nf = (int)p.pay.size() / 3, ns = (int)p.pairs.size();
                if (nf >= kRpMinRunPhases) {
                    std::vector<double> pay = p.pay;
                    pay.insert(pay.end(), p.pairs.begin(), p.pairs.end());
                    emit(RP_PH, 1, nf, ns, pay);
                } else {
                    for (int q = 0; q < nf; q++)
                        emit(RP_PH, 0, (int)p.pay[3 * q], (int)p.pay[3 * q], {p.pay[3 * q + 1], p.pay[3 * q + 2]});
                    for (int q = 0; q < ns; q += 8) {
                        const int c = std::min(8, ns - q);
                        emit(RP_NEG, c - 1, 0, 0, std::vector<double>(p.pairs.begin() + q, p.pairs.begin() + q + c));
                    }
                }
            } else if (p.type == RP_NEG) {
                emit(RP_NEG, (int)p.pairs.size() - 1, 0, 0, std::vector<double>(p.pairs.begin(), p.pairs.end()));
            } else if (p.type == RP_PARITY && p.pairs.size() == 1) {
                emit(RP_PARITY, 0, p.pairs[0] & 31, p.pairs[0] >> 5,
                     {p.e.real(), p.e.imag(), p.f.real(), p.f.imag()});
            } else if (p.type == RP_PARITY) {
                // factor for k odd patterns out of np: e^(np - k) f^k
                const int np = (int)p.pairs.size();
                std::vector<double> pay(p.pairs.begin(), p.pairs.end());
                for (int kk = 0; kk <= np; kk++) {
                    cd t = 1.0;
                    for (int j = 0; j < np; j++) t *= j < kk ? p.f : p.e;
                    pay.push_back(t.real());
                    pay.push_back(t.imag());
                }
                emit(RP_PARITYN, 0, 0, 0, pay);
            } else {
                emit(p.type, p.slot, p.ea, p.eb, p.pay);
            }
        }
        mats[(size_t)k.mat] = (double)n_emitted;
        k.nmat = (int32_t)mats.size() - k.mat;
        out.push_back(k);
        phases++;
    }
    if (n_phases) *n_phases = phases;
    return out;
}

double kop_touched_fraction(const KOp &k, int sector_bits) {
    if (k.fkind == F_DIAGK || k.fkind == F_DENSEK) return 1.0;
    // distinct touched patterns on the fixed bits at or above the sector granularity
    uint64_t hi_mask = 0;
    int nhi = 0;
    for (int j = 0; j < k.nf; j++)
        if (k.fb[j] >= sector_bits) {
            hi_mask |= 1ull << k.fb[j];
            nhi++;
        }
    uint64_t pat[4];
    int npat = 0;
    for (int t = 0; t < k.nt; t++) {
        const uint64_t p = (k.off[t] | k.set_mask) & hi_mask;
        bool seen = false;
        for (int u = 0; u < npat; u++) seen |= pat[u] == p;
        if (!seen) pat[npat++] = p;
    }
    return (double)npat / (double)(1ull << nhi);
}

double stream_bytes(const Op &op, int n, int dtype) {
    if (op.kind == K_PHASEFN) return 2.0 * (dtype == QS_C128 ? 16.0 : 8.0) * (double)(1ull << n);
    std::vector<int> ident(64);
    for (int i = 0; i < 64; i++) ident[i] = i;
    std::vector<double> mats;
    const KOp k = make_kop(op, ident.data(), mats);
    const double B = dtype == QS_C128 ? 16.0 : 8.0;
    const int sector_bits = dtype == QS_C128 ? 1 : 2;  // 32-byte DRAM sectors
    return 2.0 * B * (double)(1ull << n) * kop_touched_fraction(k, sector_bits);
}

}  // namespace qs
