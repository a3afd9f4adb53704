// Host: lowered Op -> kernel-side KOp in a given index space, plus algorithmic bytes.
#include <algorithm>
#include <cmath>

#include "kgeom.h"

namespace qs {

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
        return base(F_H, {p}, 0, {0, 1ull << p});
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

bool rg_eligible(const KOp &k) {
    switch (k.fkind) {
    case F_H: case F_SWAP: case F_DENSE1: case F_DIAG1: case F_PHASE: case F_NEG: case F_DIAG2: case F_DENSE2:
        return k.nf == 1 || k.nf == 2;
    default:
        return false;
    }
}

// The op as a dense 2^nf x 2^nf matrix on its fixed bits (sub-index bit j <-> fb[j]),
// obtained by applying it to every basis vector of one group.
std::vector<cd> member_matrix(const KOp &k, const std::vector<double> &mats) {
    const int nb = k.nf, D = 1 << nb;
    auto sub = [&](uint64_t x) {
        int s = 0;
        for (int j = 0; j < nb; j++) s |= (int)((x >> k.fb[j]) & 1ull) << j;
        return s;
    };
    auto mc = [&](int i) { return cd(mats[k.mat + 2 * i], mats[k.mat + 2 * i + 1]); };
    std::vector<cd> M((size_t)D * D, 0.0);
    for (int s0 = 0; s0 < D; s0++) {
        std::vector<cd> v(D, 0.0);
        v[s0] = 1.0;
        cd a[4];
        int idx[4];
        for (int t = 0; t < k.nt; t++) {
            idx[t] = sub(k.off[t] | k.set_mask);
            a[t] = v[idx[t]];
        }
        cd y[4];
        switch (k.fkind) {
        case F_H: {
            const double r = 1.0 / std::sqrt(2.0);
            y[0] = (a[0] + a[1]) * r;
            y[1] = (a[0] - a[1]) * r;
            break;
        }
        case F_SWAP: y[0] = a[1]; y[1] = a[0]; break;
        case F_DENSE1:
            y[0] = mc(0) * a[0] + mc(1) * a[1];
            y[1] = mc(2) * a[0] + mc(3) * a[1];
            break;
        case F_DIAG1: y[0] = mc(0) * a[0]; y[1] = mc(1) * a[1]; break;
        case F_PHASE: y[0] = mc(0) * a[0]; break;
        case F_NEG: y[0] = -a[0]; break;
        case F_DIAG2:
            for (int t = 0; t < 4; t++) y[t] = mc(t) * a[t];
            break;
        case F_DENSE2:
            for (int r = 0; r < 4; r++) {
                y[r] = 0.0;
                for (int c = 0; c < 4; c++) y[r] += mc(4 * r + c) * a[c];
            }
            break;
        default:
            break;
        }
        for (int t = 0; t < k.nt; t++) v[idx[t]] = y[t];
        for (int r = 0; r < D; r++) M[(size_t)r * D + s0] = v[r];
    }
    return M;
}

}  // namespace

std::vector<KOp> group_registers(const std::vector<KOp> &in, std::vector<double> &mats, int m) {
    if (m < 5) return in;
    std::vector<KOp> out;
    std::vector<const KOp *> members;
    uint32_t pos_mask = 0;
    int floats = 1;
    constexpr int kBudget = 500;  // block floats (kMaxOpReals = 512)
    auto flush = [&]() {
        if (members.size() >= 2) {
            KOp g{};
            g.fkind = F_RGROUP;
            g.k = 4;
            uint32_t S = pos_mask;
            for (int b = m - 1; b >= 0 && __builtin_popcount(S) < 4; b--) S |= 1u << b;  // pad from the top
            int np = 0;
            for (int b = 0; b < m; b++)
                if ((S >> b) & 1u) g.pos[np++] = b;
            g.mat = (int32_t)mats.size();
            mats.push_back((double)members.size());
            for (const KOp *k : members) {
                int bits[2] = {0, 0};
                for (int j = 0; j < k->nf; j++)
                    for (int t = 0; t < 4; t++)
                        if (g.pos[t] == k->fb[j]) bits[j] = t;
                mats.push_back((double)(k->nf + 4 * bits[0] + 16 * bits[1]));
                for (const cd &z : member_matrix(*k, mats)) {
                    mats.push_back(z.real());
                    mats.push_back(z.imag());
                }
            }
            g.nmat = (int32_t)mats.size() - g.mat;
            out.push_back(g);
        } else {
            for (const KOp *k : members) out.push_back(*k);
        }
        members.clear();
        pos_mask = 0;
        floats = 1;
    };
    for (const KOp &k : in) {
        if (!rg_eligible(k)) {
            flush();
            out.push_back(k);
            continue;
        }
        uint32_t km = 0;
        for (int j = 0; j < k.nf; j++) km |= 1u << k.fb[j];
        const int cost = 1 + 2 * (1 << (2 * k.nf));
        if (__builtin_popcount(pos_mask | km) > 4 || floats + cost > kBudget) flush();
        members.push_back(&k);
        pos_mask |= km;
        floats += cost;
    }
    flush();
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
    std::vector<int> ident(64);
    for (int i = 0; i < 64; i++) ident[i] = i;
    std::vector<double> mats;
    const KOp k = make_kop(op, ident.data(), mats);
    const double B = dtype == QS_C128 ? 16.0 : 8.0;
    const int sector_bits = dtype == QS_C128 ? 1 : 2;  // 32-byte DRAM sectors
    return 2.0 * B * (double)(1ull << n) * kop_touched_fraction(k, sector_bits);
}

}  // namespace qs
