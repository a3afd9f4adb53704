/*
 * Plain FP64 state-vector oracle.  TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the CPU-baseline leg of the benchmark call it; the product
 * library never links, loads or calls it, and it shares no code with it.
 *
 * What it computes (QueenV2, arXiv 2409.14697):
 *   - the state is 2^N complex amplitudes a_i, basis index i in [0, 2^N)  (Sec. II-A, Eq. 1);
 *     qubit q is bit q of i (little-endian: low qubits are contiguous, Sec. II-B
 *     "least significant bits");
 *   - a one-qubit gate G (2x2) replaces each pair of amplitudes that differ only
 *     in bit q by G times that pair (Eq. 2);
 *   - a k-qubit gate (2^k x 2^k) replaces each group of 2^k amplitudes that differ
 *     only in its operand bits by the matrix times the group (Sec. II-A, the
 *     generalisation stated before Eq. 3).  With operands (q_0, ..., q_{k-1}) the
 *     row/column index inside the group is s = sum_j bit(q_j) * 2^(k-1-j): the first
 *     operand is the most significant, which is the row order of Eq. 3, whose
 *     printed CNOT matrix makes the first operand the control.
 *
 * Gate matrices are not given by the paper (it gives only the CNOT matrix); the
 * oracle defines them here (H, X, Y, Z, S, T, RX, RY, RZ, P, U3, CNOT, CZ, SWAP,
 * CU3, CP, RZZ, dense) and the CPU tests pin every one of them against matrix
 * exponentials, textbook identities and Eq. 3.
 *
 * Everything is applied gate by gate, in order: no fusion, no reordering, no
 * blocking.  Sums (norm, <Z_i>) use pairwise summation.  Arithmetic is C99
 * double complex.
 *
 * Threads (OpenMP, when the compiler has it): the groups of one gate are
 * independent, so they are split over threads; each group's arithmetic is the
 * same as with one thread.  The pairwise sums hand whole subtrees of the same
 * tree to threads and add them in the same order.  Results are therefore bitwise
 * equal for every thread count (a CPU test checks this).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

/* Threads used by or_apply_matrix, or_norm and or_expz (1 without OpenMP). */
int or_set_threads(int t)
{
#ifdef _OPENMP
    g_threads = t < 1 ? 1 : t;
#else
    (void)t;
    g_threads = 1;
#endif
    return g_threads;
}

int or_get_threads(void) { return g_threads; }

/* 1 if this library was compiled with OpenMP. */
int or_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

typedef double complex cplx;

/* Gate type ids: the same numbering as the public C interface of the library
 * (an interface both sides must agree on; this file keeps its own copy). */
enum {
    OR_H = 0, OR_X = 1, OR_Y = 2, OR_Z = 3, OR_S = 4, OR_T = 5,
    OR_RX = 6, OR_RY = 7, OR_RZ = 8, OR_P = 9, OR_U3 = 10,
    OR_CNOT = 11, OR_CZ = 12, OR_SWAP = 13, OR_CU3 = 14, OR_CP = 15, OR_RZZ = 16,
    OR_DENSE = 17
};

/* Number of operand qubits of a gate type (-1: unknown, 0: given by the caller). */
int or_gate_arity(int type)
{
    switch (type) {
    case OR_H: case OR_X: case OR_Y: case OR_Z: case OR_S: case OR_T:
    case OR_RX: case OR_RY: case OR_RZ: case OR_P: case OR_U3:
        return 1;
    case OR_CNOT: case OR_CZ: case OR_SWAP: case OR_CU3: case OR_CP: case OR_RZZ:
        return 2;
    case OR_DENSE:
        return 0;
    default:
        return -1;
    }
}

/* U3(theta, phi, lambda) in the OpenQASM 2 convention:
 *   [[cos(t/2),              -e^{i lambda} sin(t/2)],
 *    [e^{i phi} sin(t/2),     e^{i(phi+lambda)} cos(t/2)]]              */
static void u3_matrix(const double *p, cplx *m)
{
    double c = cos(0.5 * p[0]), s = sin(0.5 * p[0]);
    m[0] = c;
    m[1] = -cexp(I * p[2]) * s;
    m[2] = cexp(I * p[1]) * s;
    m[3] = cexp(I * (p[1] + p[2])) * c;
}

/* Writes the gate's 2^k x 2^k matrix (row-major) to out; returns k, or -1 for an
 * unknown type.  OR_DENSE is not handled here (the caller supplies its matrix). */
int or_gate_matrix(int type, const double *p, double *out_interleaved)
{
    cplx *m = (cplx *)out_interleaved;
    const double r = 1.0 / sqrt(2.0);
    int k = or_gate_arity(type);
    if (k <= 0)
        return -1;
    memset(m, 0, sizeof(cplx) << (2 * k));
    switch (type) {
    case OR_H: m[0] = r; m[1] = r; m[2] = r; m[3] = -r; break;
    case OR_X: m[1] = 1; m[2] = 1; break;
    case OR_Y: m[1] = -I; m[2] = I; break;
    case OR_Z: m[0] = 1; m[3] = -1; break;
    case OR_S: m[0] = 1; m[3] = I; break;
    case OR_T: m[0] = 1; m[3] = cexp(I * M_PI / 4); break;
    case OR_RX: {           /* exp(-i theta X / 2) */
        double c = cos(0.5 * p[0]), s = sin(0.5 * p[0]);
        m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c;
        break;
    }
    case OR_RY: {           /* exp(-i theta Y / 2) */
        double c = cos(0.5 * p[0]), s = sin(0.5 * p[0]);
        m[0] = c; m[1] = -s; m[2] = s; m[3] = c;
        break;
    }
    case OR_RZ:             /* exp(-i theta Z / 2): the global phase is kept */
        m[0] = cexp(-0.5 * I * p[0]); m[3] = cexp(0.5 * I * p[0]);
        break;
    case OR_P: m[0] = 1; m[3] = cexp(I * p[0]); break;
    case OR_U3: u3_matrix(p, m); break;
    case OR_CNOT:           /* Eq. 3: rows 0_c0_t, 0_c1_t, 1_c0_t, 1_c1_t */
        m[0 * 4 + 0] = 1; m[1 * 4 + 1] = 1; m[2 * 4 + 3] = 1; m[3 * 4 + 2] = 1;
        break;
    case OR_CZ:
        m[0] = 1; m[5] = 1; m[10] = 1; m[15] = -1;
        break;
    case OR_SWAP:
        m[0 * 4 + 0] = 1; m[1 * 4 + 2] = 1; m[2 * 4 + 1] = 1; m[3 * 4 + 3] = 1;
        break;
    case OR_CU3: {          /* |0><0| (x) I + |1><1| (x) U3, no extra phase */
        cplx u[4];
        u3_matrix(p, u);
        m[0] = 1; m[5] = 1;
        m[2 * 4 + 2] = u[0]; m[2 * 4 + 3] = u[1];
        m[3 * 4 + 2] = u[2]; m[3 * 4 + 3] = u[3];
        break;
    }
    case OR_CP:
        m[0] = 1; m[5] = 1; m[10] = 1; m[15] = cexp(I * p[0]);
        break;
    case OR_RZZ: {          /* exp(-i theta Z(x)Z / 2) */
        cplx e = cexp(-0.5 * I * p[0]), f = cexp(0.5 * I * p[0]);
        m[0] = e; m[5] = f; m[10] = f; m[15] = e;
        break;
    }
    default:
        return -1;
    }
    return k;
}

/* Applies a k-qubit matrix U (row-major 2^k x 2^k, interleaved re/im) on
 * operands q[0..k-1] (q[0] most significant in the group index) to the
 * n-qubit state psi: for every base index x whose operand bits are all zero,
 * gather v_s = psi[x + sum_j bit_j(s) 2^q_j], form U v and scatter it back.
 * The base indices are enumerated as b = 0 .. 2^(n-k)-1 with a zero bit
 * inserted at each operand position (ascending), which lists each such x once. */
int or_apply_matrix(double *psi_interleaved, int n, int k, const int *q,
                    const double *u_interleaved)
{
    cplx *psi = (cplx *)psi_interleaved;
    const cplx *u = (const cplx *)u_interleaved;
    uint64_t opmask = 0;
    int G = 1 << k, nt = g_threads, sorted_q[12];
    int64_t n_base;
    uint64_t *off;
    cplx *vw;
    if (k < 1 || k > 12 || n < k || n > 40)
        return -1;
    for (int j = 0; j < k; j++) {
        if (q[j] < 0 || q[j] >= n || (opmask >> q[j]) & 1)
            return -1;
        opmask |= (uint64_t)1 << q[j];
    }
    for (int j = 0, c = 0; j < n; j++)
        if ((opmask >> j) & 1)
            sorted_q[c++] = j;
    n_base = (int64_t)1 << (n - k);
    off = malloc(sizeof(uint64_t) * G);
    vw = malloc(sizeof(cplx) * 2 * G * (size_t)nt);   /* v and w per thread */
    if (!off || !vw) {
        free(off); free(vw);
        return -2;
    }
    for (int s = 0; s < G; s++) {
        off[s] = 0;
        for (int j = 0; j < k; j++)
            if ((s >> (k - 1 - j)) & 1)
                off[s] |= (uint64_t)1 << q[j];
    }
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(static)
#endif
    for (int64_t b = 0; b < n_base; b++) {
        int t = 0;
        uint64_t x = (uint64_t)b;
        cplx *v, *w;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        v = vw + (size_t)2 * G * t;
        w = v + G;
        for (int j = 0; j < k; j++) {   /* insert a zero bit at sorted_q[j] */
            uint64_t lo = x & (((uint64_t)1 << sorted_q[j]) - 1);
            x = ((x >> sorted_q[j]) << (sorted_q[j] + 1)) | lo;
        }
        for (int s = 0; s < G; s++)
            v[s] = psi[x + off[s]];
        for (int r = 0; r < G; r++) {
            cplx acc = 0;
            for (int c = 0; c < G; c++)
                acc += u[r * G + c] * v[c];
            w[r] = acc;
        }
        for (int s = 0; s < G; s++)
            psi[x + off[s]] = w[s];
    }
    free(off); free(vw);
    return 0;
}

/* One gate: its matrix (own definition, or the caller's for OR_DENSE), then
 * or_apply_matrix. */
int or_apply_gate(double *psi, int n, int type, int nq, const int *q,
                  const double *p, const double *dense)
{
    int k = or_gate_arity(type);
    if (k < 0)
        return -1;
    if (type == OR_DENSE) {
        if (!dense || nq < 1)
            return -1;
        return or_apply_matrix(psi, n, nq, q, dense);
    }
    if (nq != k)
        return -1;
    {
        double m[2 * 16];
        or_gate_matrix(type, p, m);
        return or_apply_matrix(psi, n, k, q, m);
    }
}

/* A circuit of ng gates, in order.  Operands: q[g*8 + j]; angles p[g*3 + j];
 * dense matrices at dense + dense_off[g] (interleaved), ignored otherwise.
 * Returns the index+1 of the first failing gate as a negative number. */
int or_run(double *psi, int n, long ng, const int *type, const int *nq,
           const int *q, const double *p, const double *dense,
           const long *dense_off)
{
    for (long g = 0; g < ng; g++) {
        const double *dm = (type[g] == OR_DENSE && dense) ? dense + dense_off[g] : NULL;
        if (or_apply_gate(psi, n, type[g], nq[g], q + g * 8, p + g * 3, dm) != 0)
            return (int)(-(g + 1));
    }
    return 0;
}

/* |0...0>: a_0 = 1. */
void or_zero_state(double *psi, int n)
{
    memset(psi, 0, sizeof(cplx) << n);
    psi[0] = 1.0;
}

/* Pairwise sum of |a_x|^2 * w(x) over x in [lo, hi), w(x) = +1, or -1 when bit
 * `bit` of x is set (bit < 0: always +1). */
static double pw_sum(const cplx *psi, uint64_t lo, uint64_t hi, int bit)
{
    if (hi - lo <= 64) {
        double s = 0;
        for (uint64_t x = lo; x < hi; x++) {
            double pr = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
            s += (bit >= 0 && ((x >> bit) & 1)) ? -pr : pr;
        }
        return s;
    }
    {
        uint64_t mid = lo + (hi - lo) / 2;
        return pw_sum(psi, lo, mid, bit) + pw_sum(psi, mid, hi, bit);
    }
}

/* The same tree as pw_sum: ranges longer than `grain` are split at the same
 * midpoint, the left half going to another thread; the two halves are added in
 * the same order as pw_sum adds them. */
static double pw_sum_tasks(const cplx *psi, uint64_t lo, uint64_t hi, int bit, int depth)
{
    uint64_t mid;
    double a, b;
    if (depth <= 0 || hi - lo <= ((uint64_t)1 << 16))
        return pw_sum(psi, lo, hi, bit);
    mid = lo + (hi - lo) / 2;
#ifdef _OPENMP
#pragma omp task shared(a)
#endif
    a = pw_sum_tasks(psi, lo, mid, bit, depth - 1);
    b = pw_sum_tasks(psi, mid, hi, bit, depth - 1);
#ifdef _OPENMP
#pragma omp taskwait
#endif
    return a + b;
}

static double pw_sum_all(const cplx *psi, int n, int bit)
{
    double r = 0;
    if (g_threads <= 1)
        return pw_sum(psi, 0, (uint64_t)1 << n, bit);
#ifdef _OPENMP
#pragma omp parallel num_threads(g_threads)
#pragma omp single
#endif
    r = pw_sum_tasks(psi, 0, (uint64_t)1 << n, bit, 12);
    return r;
}

/* Squared norm sum_x |a_x|^2. */
double or_norm(const double *psi, int n)
{
    return pw_sum_all((const cplx *)psi, n, -1);
}

/* <psi| Z_i |psi> = sum_x |a_x|^2 (1 - 2 bit_i(x)) for i = 0..n-1 (not divided by
 * the norm). */
void or_expz(const double *psi, int n, double *out)
{
    for (int i = 0; i < n; i++)
        out[i] = pw_sum_all((const cplx *)psi, n, i);
}

static const cplx *g_sort_psi;

static int cmp_prob_desc(const void *a, const void *b)
{
    uint64_t i = *(const uint64_t *)a, j = *(const uint64_t *)b;
    double pi = creal(g_sort_psi[i]) * creal(g_sort_psi[i]) + cimag(g_sort_psi[i]) * cimag(g_sort_psi[i]);
    double pj = creal(g_sort_psi[j]) * creal(g_sort_psi[j]) + cimag(g_sort_psi[j]) * cimag(g_sort_psi[j]);
    if (pi > pj) return -1;
    if (pi < pj) return 1;
    return (i < j) ? -1 : (i > j);
}

/* The k amplitudes of largest |a|^2, ties broken by the lower index; writes
 * indices and interleaved amplitudes.  Sorts all 2^n indices (plain, slow). */
int or_top_k(const double *psi, int n, long k, uint64_t *idx, double *amp)
{
    uint64_t dim = (uint64_t)1 << n;
    uint64_t *ord;
    if (k < 0 || (uint64_t)k > dim)
        return -1;
    ord = malloc(sizeof(uint64_t) * dim);
    if (!ord)
        return -2;
    for (uint64_t x = 0; x < dim; x++)
        ord[x] = x;
    g_sort_psi = (const cplx *)psi;
    qsort(ord, dim, sizeof(uint64_t), cmp_prob_desc);
    for (long t = 0; t < k; t++) {
        idx[t] = ord[t];
        amp[2 * t] = psi[2 * ord[t]];
        amp[2 * t + 1] = psi[2 * ord[t] + 1];
    }
    free(ord);
    return 0;
}
