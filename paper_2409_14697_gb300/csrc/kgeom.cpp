// Host: lowered Op -> kernel-side KOp in a given index space, plus algorithmic bytes.
#include <algorithm>

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
