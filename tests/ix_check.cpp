// Test program (built and run by tests/test_ix_cpu.py, CPU only): the integer-product
// arithmetic of complex128 streaming updates (csrc/ixmath.cuh, host build of the same
// functions the kernels run) against exact sums in binary128.
//
// For seeded random terms and one-qubit updates (Eq. 2: U3-class, general unitary, real
// (RY) and RX-class 2x2 matrices, diagonal phases) on amplitudes of several magnitude profiles (Gaussian state
// amplitudes, independent exponents over 80 binades, exact zeros, structured values):
//   * both result encodings (integer-to-double conversion, integer instructions only)
//     give the same bits;
//   * every output is within 0.5 ulp + 2^-56.4 max_k |c_k x_k| of the exact sum;
//   * the largest error, in units of max_k |c_k x_k|, is no larger than that of the
//     native FP64 multiply-add chains the FP64 kernels run (kops.cuh), and the count of
//     outputs where the integer form is further from the exact value than native FP64 is
//     printed.
// Usage: ix_check <seed> <trials>; prints OK and statistics, exits 0 on success.
//        ix_check --apply <r0|gen|real|rx|phase> <n> <q> <state.bin> <matrix.bin> <out.bin>:
//        applies one gate on qubit q of a 2^n complex128 state in the integer form, every
//        group (phase: the elements whose bit q is 1 times the factor m[0] + i m[1]; the
//        others: the 2x2 matrix m[8] on every pair, in the 14-term form with a real first
//        entry, the general 16-term form, the real form or the RX form), and writes the
//        resulting state.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "ixmath.cuh"

#if defined(__x86_64__) || defined(__i386__)
typedef __float128 Q;
#else
static_assert(LDBL_MANT_DIG >= 113, "needs a binary128 long double");
typedef long double Q;
#endif

using qs::ix::Num;

static int g_fail = 0;
static long g_outputs = 0, g_worse = 0;
static double g_max_ix = 0, g_max_nat = 0;

static double qabs(Q v) { return (double)(v < 0 ? -v : v); }

// ulp of the double nearest to v (normal range)
static double ulp_of(double v) {
    if (v == 0) return 0x1p-1074;
    int e;
    std::frexp(std::fabs(v), &e);
    return std::ldexp(1.0, e - 53);
}

// One output: exact sum of terms (value, coefficient, sign) against both forms.
struct Term {
    double x, c;
    bool neg;
};

static void check_output(const char *what, double got_cvt, double got_int, double native, const Term *t, int k) {
    Q exact = 0;
    double maxterm = 0;
    for (int i = 0; i < k; i++) {
        Q p = (Q)t[i].x * (Q)t[i].c;  // exact: 53 x 53 bits fit binary128
        if (t[i].neg) p = -p;
        exact += p;
        maxterm = std::fmax(maxterm, std::fabs(t[i].x * t[i].c));
    }
    g_outputs++;
    uint64_t a = qs::ix::bits_of(got_cvt), b = qs::ix::bits_of(got_int);
    if (a != b) {
        if (g_fail++ < 10) std::printf("FAIL %s: encodings differ %.17g %.17g\n", what, got_cvt, got_int);
        return;
    }
    const double err = qabs((Q)got_cvt - exact);
    const double errn = qabs((Q)native - exact);
    const double ex = (double)exact;
    const double bound = 0.5 * ulp_of(ex) + std::ldexp(maxterm, -56) * 0.75;  // 2^-56.4 < 0.76 * 2^-56
    // flushed tiny outputs (unit below 2^-1022) are not checked against the bound
    if (maxterm > 0x1p-900 && err > bound) {
        if (g_fail++ < 10)
            std::printf("FAIL %s: err %.3e > bound %.3e (exact %.17g got %.17g maxterm %.3e)\n", what, err, bound,
                        ex, got_cvt, maxterm);
    }
    if (maxterm > 0x1p-900) {
        g_max_ix = std::fmax(g_max_ix, err / maxterm);
        g_max_nat = std::fmax(g_max_nat, errn / maxterm);
        if (err > errn) g_worse++;
    }
}

// random double with the given binade range [lo, hi) and random sign
static double rnd_mag(std::mt19937_64 &r, int lo, int hi) {
    std::uniform_real_distribution<double> u(1.0, 2.0);
    std::uniform_int_distribution<int> e(lo, hi - 1);
    double v = std::ldexp(u(r), e(r));
    return (r() & 1) ? -v : v;
}

static double amp_value(std::mt19937_64 &r, int profile) {
    std::normal_distribution<double> g(0.0, std::ldexp(1.0, -15));
    switch (profile) {
    case 0: return g(r);                                   // Gaussian state amplitude
    case 1: return rnd_mag(r, -80, 0);                     // wide independent exponents
    case 2: return (r() % 3 == 0) ? 0.0 : g(r);            // exact zeros
    case 3: return (r() & 1 ? 1 : -1) * std::sqrt(0.5) * std::ldexp(1.0, -(int)(r() % 4));  // structured
    default: return rnd_mag(r, -1000, -960);                // near the flush range
    }
}

// native FP64 chains as the FP64 kernels evaluate them (kops.cuh)
static void native_r0(const double *m, const double *x, double *y) {
    const double ar = x[0], ai = x[1], br = x[2], bi = x[3];
    double pr = m[2] * br;
    pr = std::fma(-m[3], bi, pr);
    double pi = m[2] * bi;
    pi = std::fma(m[3], br, pi);
    double yr = m[4] * ar;
    yr = std::fma(-m[5], ai, yr);
    yr = std::fma(m[6], br, yr);
    yr = std::fma(-m[7], bi, yr);
    double yi = m[4] * ai;
    yi = std::fma(m[5], ar, yi);
    yi = std::fma(m[6], bi, yi);
    yi = std::fma(m[7], br, yi);
    y[0] = std::fma(m[0], ar, pr);
    y[1] = std::fma(m[0], ai, pi);
    y[2] = yr;
    y[3] = yi;
}

static void native_general(const double *m, const double *x, double *y) {
    for (int row = 0; row < 2; row++) {
        const double *q = m + 4 * row;
        double yr = q[0] * x[0];
        yr = std::fma(-q[1], x[1], yr);
        yr = std::fma(q[2], x[2], yr);
        yr = std::fma(-q[3], x[3], yr);
        double yi = q[0] * x[1];
        yi = std::fma(q[1], x[0], yi);
        yi = std::fma(q[2], x[3], yi);
        yi = std::fma(q[3], x[2], yi);
        y[2 * row] = yr;
        y[2 * row + 1] = yi;
    }
}

static void u3(double th, double ph, double la, double *m) {
    const double c = std::cos(th / 2), s = std::sin(th / 2);
    m[0] = c; m[1] = 0;
    m[2] = -std::cos(la) * s; m[3] = -std::sin(la) * s;
    m[4] = std::cos(ph) * s; m[5] = std::sin(ph) * s;
    m[6] = std::cos(ph + la) * c; m[7] = std::sin(ph + la) * c;
}

static int apply_file(int argc, char **argv) {
    if (argc != 8) {
        std::printf("usage: ix_check --apply <r0|gen|phase> <n> <q> <state> <matrix> <out>\n");
        return 2;
    }
    const std::string kind = argv[2];
    const int n = std::atoi(argv[3]), q = std::atoi(argv[4]);
    const size_t dim = (size_t)1 << n;
    std::vector<double> psi(2 * dim), m(8, 0.0);
    FILE *f = std::fopen(argv[5], "rb");
    if (!f || std::fread(psi.data(), 16, dim, f) != dim) return 3;
    std::fclose(f);
    f = std::fopen(argv[6], "rb");
    const size_t nm = kind == "phase" ? 2 : 8;
    if (!f || std::fread(m.data(), 8, nm, f) != nm) return 3;
    std::fclose(f);
    Num c[16];
    if (kind == "phase") qs::ix::rows_diag(c, m.data(), 1);
    else if (kind == "real") qs::ix::rows_dense1_real(c, m.data());
    else if (kind == "rx") qs::ix::rows_dense1_rx(c, m.data());
    else qs::ix::rows_dense1(c, m.data(), kind == "r0");
    for (size_t i = 0; i < dim; i++) {
        if ((i >> q) & 1) continue;
        const size_t j = i | ((size_t)1 << q);
        if (kind == "phase") {
            const Num x[2] = {qs::ix::decode(psi[2 * j]), qs::ix::decode(psi[2 * j + 1])};
            double y[2];
            qs::ix::phase<2>(c, x, y);
            psi[2 * j] = y[0];
            psi[2 * j + 1] = y[1];
            continue;
        }
        const Num x[4] = {qs::ix::decode(psi[2 * i]), qs::ix::decode(psi[2 * i + 1]),
                          qs::ix::decode(psi[2 * j]), qs::ix::decode(psi[2 * j + 1])};
        double y[4];
        if (kind == "r0") qs::ix::dense1_r0<2>(c, x, y);
        else if (kind == "real") qs::ix::dense1_real<2>(c, x, y);
        else if (kind == "rx") qs::ix::dense1_rx<2>(c, x, y);
        else qs::ix::dense1<2>(c, x, y);
        psi[2 * i] = y[0]; psi[2 * i + 1] = y[1];
        psi[2 * j] = y[2]; psi[2 * j + 1] = y[3];
    }
    f = std::fopen(argv[7], "wb");
    if (!f || std::fwrite(psi.data(), 16, dim, f) != dim) return 3;
    std::fclose(f);
    return 0;
}

int main(int argc, char **argv) {
    if (argc > 1 && std::string(argv[1]) == "--apply") return apply_file(argc, argv);
    const unsigned long seed = argc > 1 ? std::strtoul(argv[1], nullptr, 10) : 1;
    const long trials = argc > 2 ? std::strtol(argv[2], nullptr, 10) : 100000;
    std::mt19937_64 r(seed);
    std::uniform_real_distribution<double> ang(0.0, 2 * M_PI);

    for (long t = 0; t < trials; t++) {
        const int profile = (int)(t % 5);
        double x[4];
        for (int i = 0; i < 4; i++) x[i] = amp_value(r, profile);
        Num nx[4];
        for (int i = 0; i < 4; i++) nx[i] = qs::ix::decode(x[i]);

        // U3 class (14 terms); every few trials a near-identity or tiny-angle matrix
        double m[8];
        const double th = (t % 7 == 0) ? std::ldexp(ang(r), -(int)(r() % 40)) : ang(r);
        u3(th, ang(r), ang(r), m);
        {
            Num c[14];
            qs::ix::rows_dense1(c, m, true);
            double yc[4], yi[4], yn[4];
            qs::ix::dense1_r0<0>(c, nx, yc);
            qs::ix::dense1_r0<2>(c, nx, yi);
            native_r0(m, x, yn);
            const Term t0[3] = {{x[0], m[0], false}, {x[2], m[2], false}, {x[3], m[3], true}};
            const Term t1[3] = {{x[1], m[0], false}, {x[3], m[2], false}, {x[2], m[3], false}};
            const Term t2[4] = {{x[0], m[4], false}, {x[1], m[5], true}, {x[2], m[6], false}, {x[3], m[7], true}};
            const Term t3[4] = {{x[1], m[4], false}, {x[0], m[5], false}, {x[3], m[6], false}, {x[2], m[7], false}};
            check_output("u3 re a", yc[0], yi[0], yn[0], t0, 3);
            check_output("u3 im a", yc[1], yi[1], yn[1], t1, 3);
            check_output("u3 re b", yc[2], yi[2], yn[2], t2, 4);
            check_output("u3 im b", yc[3], yi[3], yn[3], t3, 4);
        }
        // general unitary: U3 times a global phase (Im m00 != 0)
        {
            const double g = ang(r), cg = std::cos(g), sg = std::sin(g);
            double q[8];
            for (int i = 0; i < 4; i++) {
                q[2 * i] = m[2 * i] * cg - m[2 * i + 1] * sg;
                q[2 * i + 1] = m[2 * i] * sg + m[2 * i + 1] * cg;
            }
            Num c[16];
            qs::ix::rows_dense1(c, q, false);
            double yc[4], yi[4], yn[4];
            qs::ix::dense1<0>(c, nx, yc);
            qs::ix::dense1<2>(c, nx, yi);
            native_general(q, x, yn);
            for (int row = 0; row < 2; row++) {
                const double *p = q + 4 * row;
                const Term tr[4] = {{x[0], p[0], false}, {x[1], p[1], true}, {x[2], p[2], false}, {x[3], p[3], true}};
                const Term ti[4] = {{x[1], p[0], false}, {x[0], p[1], false}, {x[3], p[2], false}, {x[2], p[3], false}};
                check_output("general re", yc[2 * row], yi[2 * row], yn[2 * row], tr, 4);
                check_output("general im", yc[2 * row + 1], yi[2 * row + 1], yn[2 * row + 1], ti, 4);
            }
        }
        // real rotation (RY class) and RX class: rows of 2 terms
        {
            const double a = ang(r) / 2, ca = std::cos(a), sa = std::sin(a);
            const double ry[8] = {ca, 0, -sa, 0, sa, 0, ca, 0};
            const double rx[8] = {ca, 0, 0, -sa, 0, -sa, ca, 0};
            Num c[8];
            double yc[4], yi[4];
            qs::ix::rows_dense1_real(c, ry);
            qs::ix::dense1_real<0>(c, nx, yc);
            qs::ix::dense1_real<2>(c, nx, yi);
            const double nry[4] = {std::fma(ry[0], x[0], ry[2] * x[2]), std::fma(ry[0], x[1], ry[2] * x[3]),
                                   std::fma(ry[4], x[0], ry[6] * x[2]), std::fma(ry[4], x[1], ry[6] * x[3])};
            const Term a0[2] = {{x[0], ry[0], false}, {x[2], ry[2], false}};
            const Term a1[2] = {{x[1], ry[0], false}, {x[3], ry[2], false}};
            const Term b0[2] = {{x[0], ry[4], false}, {x[2], ry[6], false}};
            const Term b1[2] = {{x[1], ry[4], false}, {x[3], ry[6], false}};
            check_output("ry re a", yc[0], yi[0], nry[0], a0, 2);
            check_output("ry im a", yc[1], yi[1], nry[1], a1, 2);
            check_output("ry re b", yc[2], yi[2], nry[2], b0, 2);
            check_output("ry im b", yc[3], yi[3], nry[3], b1, 2);
            qs::ix::rows_dense1_rx(c, rx);
            qs::ix::dense1_rx<0>(c, nx, yc);
            qs::ix::dense1_rx<2>(c, nx, yi);
            const double nrx[4] = {std::fma(rx[0], x[0], -rx[3] * x[3]), std::fma(rx[0], x[1], rx[3] * x[2]),
                                   std::fma(rx[6], x[2], -rx[5] * x[1]), std::fma(rx[6], x[3], rx[5] * x[0])};
            const Term c0[2] = {{x[0], rx[0], false}, {x[3], rx[3], true}};
            const Term c1[2] = {{x[1], rx[0], false}, {x[2], rx[3], false}};
            const Term d0[2] = {{x[2], rx[6], false}, {x[1], rx[5], true}};
            const Term d1[2] = {{x[3], rx[6], false}, {x[0], rx[5], false}};
            check_output("rx re a", yc[0], yi[0], nrx[0], c0, 2);
            check_output("rx im a", yc[1], yi[1], nrx[1], c1, 2);
            check_output("rx re b", yc[2], yi[2], nrx[2], d0, 2);
            check_output("rx im b", yc[3], yi[3], nrx[3], d1, 2);
        }
        // diagonal factor
        {
            const double a = ang(r);
            const double d[2] = {std::cos(a), std::sin(a)};
            Num c[4];
            qs::ix::rows_diag(c, d, 1);
            const Num px[2] = {nx[0], nx[1]};
            double yc[2], yi[2];
            qs::ix::phase<0>(c, px, yc);
            qs::ix::phase<2>(c, px, yi);
            double yt[2];  // the same factor decoded per amplitude (diagonal tables)
            qs::ix::cmul<0>(d[0], d[1], px, yt);
            if (qs::ix::bits_of(yt[0]) != qs::ix::bits_of(yc[0]) || qs::ix::bits_of(yt[1]) != qs::ix::bits_of(yc[1])) {
                if (g_fail++ < 10) std::printf("FAIL table factor form differs\n");
            }
            const double nr = std::fma(d[0], x[0], -d[1] * x[1]);
            const double ni = std::fma(d[0], x[1], d[1] * x[0]);
            const Term tr[2] = {{x[0], d[0], false}, {x[1], d[1], true}};
            const Term ti[2] = {{x[1], d[0], false}, {x[0], d[1], false}};
            check_output("phase re", yc[0], yi[0], nr, tr, 2);
            check_output("phase im", yc[1], yi[1], ni, ti, 2);
        }
    }
    // exact special cases: zeros give zeros, a pure permutation is exact
    {
        const double m[8] = {0, 0, 1, 0, 1, 0, 0, 0};  // X
        Num c[16];
        qs::ix::rows_dense1(c, m, false);
        const double x[4] = {0.25, -0.5, 0x1.23456789abcdefp-20, -0x1.fedcba987654p-3};
        Num nx[4];
        for (int i = 0; i < 4; i++) nx[i] = qs::ix::decode(x[i]);
        double y[4];
        qs::ix::dense1<0>(c, nx, y);
        if (y[0] != x[2] || y[1] != x[3] || y[2] != x[0] || y[3] != x[1]) {
            std::printf("FAIL X is not exact\n");
            g_fail++;
        }
        const Num z[4] = {qs::ix::decode(0.0), qs::ix::decode(-0.0), qs::ix::decode(0.0), qs::ix::decode(0.0)};
        qs::ix::dense1<2>(c, z, y);
        if (y[0] != 0 || y[1] != 0 || y[2] != 0 || y[3] != 0) {
            std::printf("FAIL zeros do not stay zero\n");
            g_fail++;
        }
    }
    std::printf("outputs %ld max_err_ix %.3e max_err_native %.3e (units of the largest term) ix_worse %ld\n",
                g_outputs, g_max_ix, g_max_nat, g_worse);
    if (g_max_ix > g_max_nat) {
        std::printf("FAIL the integer form's largest error exceeds native FP64's\n");
        g_fail++;
    }
    if (g_fail) return 1;
    std::printf("OK\n");
    return 0;
}
