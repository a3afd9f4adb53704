// Host side of merged diagonal runs: exact decomposition of each diagonal gate, grouping of
// equal factors, and the combined phase table (FP64).
#include "phasefn.h"

#include <algorithm>
#include <map>

namespace qs {

namespace {

// The 2x2-qubit diagonal of op in (first operand, second operand) order: d[2 x_a + x_b];
// one-qubit diagonals use a = b (entries d0 = d(0), d3 = d(1)).
bool diag_entries(const Op &op, int &a, int &b, cd (&d)[4]) {
    switch (op.kind) {
    case K_DIAG1:
        a = b = op.q[0];
        d[0] = op.m[0];
        d[3] = op.m[1];
        return true;
    case K_DIAG:
        if (op.k == 1) {
            a = b = op.q[0];
            d[0] = op.m[0];
            d[3] = op.m[1];
            return true;
        }
        if (op.k != 2) return false;
        a = op.q[0];
        b = op.q[1];
        for (int i = 0; i < 4; i++) d[i] = op.m[i];
        return true;
    case K_CTRL1:
        if (op.m[1] != cd(0.0) || op.m[2] != cd(0.0)) return false;
        a = op.q[0];
        b = op.q[1];
        d[0] = 1.0;
        d[1] = 1.0;
        d[2] = op.m[0];
        d[3] = op.m[3];
        return true;
    default:
        return false;
    }
}

bool nonzero_entries(const cd (&d)[4], bool one_qubit) {
    if (one_qubit) return d[0] != cd(0.0) && d[3] != cd(0.0);
    for (const cd &z : d)
        if (z == cd(0.0)) return false;
    return true;
}

cd ipow(cd z, int k) {
    cd r = 1.0;
    for (int i = 0; i < k; i++) r *= z;
    return r;
}

// std::complex has no ordering; key factors by their bit patterns.
struct CdKey {
    double re, im;
    bool operator<(const CdKey &o) const { return re < o.re || (re == o.re && im < o.im); }
};

}  // namespace

bool pf_absorbs(const Op &op) {
    int a, b;
    cd d[4];
    return diag_entries(op, a, b, d) && nonzero_entries(d, a == b);
}

std::shared_ptr<const PhaseFn> build_phasefn(const std::vector<Op> &ops, size_t begin, size_t end) {
    cd C = 1.0;
    std::map<int, cd> beta;                     // per qubit
    std::map<std::pair<int, int>, cd> delta;    // per unordered pair (lo, hi)
    uint64_t qmask = 0;
    for (size_t i = begin; i < end; i++) {
        int a, b;
        cd d[4];
        if (!diag_entries(ops[i], a, b, d) || !nonzero_entries(d, a == b)) return nullptr;
        qmask |= (1ull << a) | (1ull << b);
        if (a == b) {
            C *= d[0];
            beta.emplace(a, 1.0).first->second *= d[3] / d[0];
            continue;
        }
        C *= d[0];
        beta.emplace(a, 1.0).first->second *= d[2] / d[0];
        beta.emplace(b, 1.0).first->second *= d[1] / d[0];
        delta.emplace(std::make_pair(std::min(a, b), std::max(a, b)), 1.0).first->second *=
            d[3] * d[0] / (d[1] * d[2]);
    }
    auto pf = std::make_shared<PhaseFn>();
    pf->qmask = qmask;
    // weight groups: qubits with equal beta (beta = 1 contributes nothing)
    std::map<CdKey, uint64_t> wmask;
    for (const auto &kv : beta)
        if (kv.second != cd(1.0)) wmask[{kv.second.real(), kv.second.imag()}] |= 1ull << kv.first;
    // pair groups: pairs with equal delta
    std::map<CdKey, std::vector<std::pair<int, int>>> pgroups;
    for (const auto &kv : delta)
        if (kv.second != cd(1.0)) pgroups[{kv.second.real(), kv.second.imag()}].push_back(kv.first);
    std::vector<PfGroup> groups;
    for (const auto &kv : wmask) {
        PfGroup g;
        g.kind = PF_WEIGHT;
        g.mask = kv.second;
        g.value = cd(kv.first.re, kv.first.im);
        g.max_count = __builtin_popcountll(g.mask);
        groups.push_back(g);
    }
    for (auto &kv : pgroups) {
        const std::vector<std::pair<int, int>> &pairs = kv.second;
        const cd dv(kv.first.re, kv.first.im);
        // a clique (every pair of its qubit set): count = w (w - 1) / 2 with w = popcount
        uint64_t S = 0;
        for (const auto &p : pairs) S |= (1ull << p.first) | (1ull << p.second);
        const uint64_t w = (uint64_t)__builtin_popcountll(S);
        if (w >= 3 && pairs.size() == w * (w - 1) / 2) {
            bool folded = false;
            for (PfGroup &g : groups)
                if (g.kind == PF_WEIGHT && g.mask == S && g.clique == cd(1.0)) {
                    g.clique = dv;
                    folded = true;
                    break;
                }
            if (!folded) {
                PfGroup g;
                g.kind = PF_WEIGHT;
                g.mask = S;
                g.value = 1.0;
                g.clique = dv;
                g.max_count = (int)w;
                groups.push_back(g);
            }
            continue;
        }
        PfGroup g;
        g.kind = PF_PAIRS;
        g.pairs = pairs;
        g.value = dv;
        g.max_count = (int)pairs.size();
        groups.push_back(g);
    }
    if ((int)groups.size() > kPfMaxGroups) return nullptr;
    size_t size = 1;
    for (PfGroup &g : groups) {
        g.stride = (int)size;
        size *= (size_t)(g.max_count + 1);
        if (size > (size_t)kPfMaxTable) return nullptr;
    }
    pf->table.assign(size, C);
    for (size_t idx = 0; idx < size; idx++) {
        size_t rest = idx;
        for (const PfGroup &g : groups) {
            const int c = (int)(rest % (size_t)(g.max_count + 1));
            rest /= (size_t)(g.max_count + 1);
            pf->table[idx] *= ipow(g.value, c);
            if (g.kind == PF_WEIGHT && g.clique != cd(1.0)) pf->table[idx] *= ipow(g.clique, c * (c - 1) / 2);
        }
    }
    pf->groups = std::move(groups);
    return pf;
}

std::vector<Op> merge_diagonal_runs(const std::vector<Op> &ops, int min_run,
                                    std::vector<std::pair<size_t, size_t>> *origin) {
    std::vector<Op> out;
    if (origin) origin->clear();
    size_t i = 0;
    while (i < ops.size()) {
        size_t j = i;
        while (j < ops.size() && pf_absorbs(ops[j])) j++;
        if ((int)(j - i) >= min_run) {
            std::shared_ptr<const PhaseFn> pf = build_phasefn(ops, i, j);
            if (pf) {
                Op op;
                op.kind = K_PHASEFN;
                op.k = 0;
                op.pf = pf;
                op.wide_mask = pf->qmask;
                out.push_back(std::move(op));
                if (origin) origin->emplace_back(i, j);
                i = j;
                continue;
            }
        }
        for (size_t t = i; t < std::max(j, i + 1); t++) {
            out.push_back(ops[t]);
            if (origin) origin->emplace_back(t, t + 1);
        }
        i = std::max(j, i + 1);
    }
    return out;
}

}  // namespace qs
