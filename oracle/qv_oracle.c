/*
 * CPU oracle for the state-vector hot path (test infrastructure).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may load
 * this library. It shares no code with the CUDA path. Everything is complex128
 * (C99 "double complex") with plain sequential loops, written so that each step
 * can be checked by eye against the paper:
 *
 *   - a state of n qubits is 2^n complex amplitudes (Sec. II, Eq. 1-2);
 *   - qubit k is bit k of the amplitude index (the 2^k in Eq. 5);
 *   - a single-qubit gate U on qubit k updates every pair (i, i XOR 2^k) whose
 *     index i has bit k equal to 0, once, in one scan (Sec. III-A, Eq. 5);
 *   - a controlled gate applies Eq. 5 only to pairs whose control bit is 1
 *     (the paper names CNOT but prints no rule: Sec. II mentions it next to
 *     Eq. 3; this is the textbook definition |0><0| (x) I + |1><1| (x) U);
 *   - gate matrices follow the OpenQASM definitions (the paper defines none).
 *
 * Reductions are plain FP64 sums over the whole vector. Nothing here is
 * blocked, fused or reordered.
 *
 * Built with -fopenmp, the pair loops of Eq. 5 (and the swap and permutation
 * loops) split their index range over threads. Each pair is still visited by
 * exactly one iteration, with the same arithmetic in the same order, so the
 * resulting state is bit-identical to the serial build (pinned by a test).
 * The sums of the reductions stay sequential; <Z_q> runs its n independent
 * sums on separate threads, each in index order.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Loops over fewer indices than this stay on one thread (a parallel region */
/* costs more than the loop on small states).                               */
#define ORC_PAR_MIN ((uint64_t)1 << 14)

/* Threads the parallel loops use (1 = serial); returns the number in effect. */
int orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* Gate kinds (this file's own numbering). */
enum {
    ORC_H = 0, ORC_X, ORC_Y, ORC_Z, ORC_S, ORC_SDG, ORC_T, ORC_TDG,
    ORC_RX, ORC_RY, ORC_RZ, ORC_P, ORC_U3, ORC_MATRIX, ORC_SWAP
};

typedef struct {
    int32_t kind;
    int32_t target;
    int32_t target2;   /* second qubit of SWAP, else -1 */
    int32_t ctrl;      /* control qubit, or -1 */
    double theta[3];
    double m[8];       /* MATRIX: re/im of U00, U01, U10, U11 */
} orc_gate;

/* ------------------------------------------------------------------------- */
/* Gate matrices, row-major U[0]=U00, U[1]=U01, U[2]=U10, U[3]=U11.           */
/* Row/column 0 is the amplitude whose target bit is 0.                       */
/* ------------------------------------------------------------------------- */
int orc_gate_matrix(const orc_gate *g, cplx U[4])
{
    const double th = g->theta[0], ph = g->theta[1], la = g->theta[2];
    const double r2 = 1.0 / sqrt(2.0);
    switch (g->kind) {
    case ORC_H:   U[0] = r2; U[1] = r2; U[2] = r2; U[3] = -r2; return 0;
    case ORC_X:   U[0] = 0; U[1] = 1; U[2] = 1; U[3] = 0; return 0;
    case ORC_Y:   U[0] = 0; U[1] = -I; U[2] = I; U[3] = 0; return 0;
    case ORC_Z:   U[0] = 1; U[1] = 0; U[2] = 0; U[3] = -1; return 0;
    case ORC_S:   U[0] = 1; U[1] = 0; U[2] = 0; U[3] = I; return 0;
    case ORC_SDG: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = -I; return 0;
    case ORC_T:   U[0] = 1; U[1] = 0; U[2] = 0; U[3] = cexp(I * M_PI / 4); return 0;
    case ORC_TDG: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = cexp(-I * M_PI / 4); return 0;
    case ORC_RX: /* exp(-i th X / 2) */
        U[0] = cos(th / 2); U[1] = -I * sin(th / 2);
        U[2] = -I * sin(th / 2); U[3] = cos(th / 2); return 0;
    case ORC_RY: /* exp(-i th Y / 2) */
        U[0] = cos(th / 2); U[1] = -sin(th / 2);
        U[2] = sin(th / 2); U[3] = cos(th / 2); return 0;
    case ORC_RZ: /* exp(-i th Z / 2) */
        U[0] = cexp(-I * th / 2); U[1] = 0; U[2] = 0; U[3] = cexp(I * th / 2); return 0;
    case ORC_P:
        U[0] = 1; U[1] = 0; U[2] = 0; U[3] = cexp(I * th); return 0;
    case ORC_U3: /* OpenQASM U(theta, phi, lambda) */
        U[0] = cos(th / 2);
        U[1] = -cexp(I * la) * sin(th / 2);
        U[2] = cexp(I * ph) * sin(th / 2);
        U[3] = cexp(I * (ph + la)) * cos(th / 2);
        return 0;
    case ORC_MATRIX:
        for (int e = 0; e < 4; ++e) U[e] = g->m[2 * e] + I * g->m[2 * e + 1];
        return 0;
    default:
        return -1;
    }
}

/* ------------------------------------------------------------------------- */
/* Eq. 5: scan i = 0 .. 2^n - 1; when bit k of i is 0, i is paired with       */
/* j = i XOR 2^k and (a_i, a_j) <- U (a_i, a_j). Every pair is visited once.  */
/* ------------------------------------------------------------------------- */
void orc_apply_1q(cplx *psi, int n, int k, const cplx U[4])
{
    const uint64_t dim = (uint64_t)1 << n;
    const uint64_t bit = (uint64_t)1 << k;
#pragma omp parallel for schedule(static) if (dim >= ORC_PAR_MIN)
    for (uint64_t i = 0; i < dim; ++i) {
        if (i & bit) continue;
        const uint64_t j = i ^ bit;
        const cplx a = psi[i], b = psi[j];
        psi[i] = U[0] * a + U[1] * b;
        psi[j] = U[2] * a + U[3] * b;
    }
}

/* Controlled U: Eq. 5 on the pairs (i, i XOR 2^t) with bit t of i = 0 and    */
/* bit c of i = 1; amplitudes whose control bit is 0 are left alone.          */
void orc_apply_controlled(cplx *psi, int n, int c, int t, const cplx U[4])
{
    const uint64_t dim = (uint64_t)1 << n;
    const uint64_t tbit = (uint64_t)1 << t, cbit = (uint64_t)1 << c;
#pragma omp parallel for schedule(static) if (dim >= ORC_PAR_MIN)
    for (uint64_t i = 0; i < dim; ++i) {
        if (i & tbit) continue;
        if (!(i & cbit)) continue;
        const uint64_t j = i ^ tbit;
        const cplx a = psi[i], b = psi[j];
        psi[i] = U[0] * a + U[1] * b;
        psi[j] = U[2] * a + U[3] * b;
    }
}

/* SWAP(a, b): exchange the amplitudes whose bits a and b differ. */
void orc_apply_swap(cplx *psi, int n, int a, int b)
{
    const uint64_t dim = (uint64_t)1 << n;
    const uint64_t ba = (uint64_t)1 << a, bb = (uint64_t)1 << b;
#pragma omp parallel for schedule(static) if (dim >= ORC_PAR_MIN)
    for (uint64_t i = 0; i < dim; ++i) {
        if ((i & ba) && !(i & bb)) {
            const uint64_t j = (i ^ ba) | bb;
            const cplx tmp = psi[i];
            psi[i] = psi[j];
            psi[j] = tmp;
        }
    }
}

/* Returns 0, or -1 for a bad gate (unknown kind, qubit out of range, control */
/* equal to target).                                                           */
int orc_apply_gate(cplx *psi, int n, const orc_gate *g)
{
    if (g->target < 0 || g->target >= n) return -1;
    if (g->kind == ORC_SWAP) {
        if (g->target2 < 0 || g->target2 >= n || g->target2 == g->target) return -1;
        orc_apply_swap(psi, n, g->target, g->target2);
        return 0;
    }
    cplx U[4];
    if (orc_gate_matrix(g, U)) return -1;
    if (g->ctrl < 0) {
        orc_apply_1q(psi, n, g->target, U);
        return 0;
    }
    if (g->ctrl >= n || g->ctrl == g->target) return -1;
    orc_apply_controlled(psi, n, g->ctrl, g->target, U);
    return 0;
}

/* Applies gates in list order (Eq. 3 once per gate). Returns the index of the */
/* first bad gate + 1, or 0.                                                   */
int64_t orc_run(cplx *psi, int n, const orc_gate *g, int64_t ng)
{
    for (int64_t l = 0; l < ng; ++l)
        if (orc_apply_gate(psi, n, &g[l])) return l + 1;
    return 0;
}

/* |j>: all amplitudes 0 except amplitude j = 1. */
void orc_basis(cplx *psi, int n, uint64_t j)
{
    const uint64_t dim = (uint64_t)1 << n;
#pragma omp parallel for schedule(static) if (dim >= ORC_PAR_MIN)
    for (uint64_t i = 0; i < dim; ++i) psi[i] = 0;
    psi[j] = 1;
}

/* Qubit permutation: bit q of the input index becomes bit perm[q] of the     */
/* output index, out[pi(i)] = in[i].                                          */
void orc_permute(const cplx *in, cplx *out, int n, const int32_t *perm)
{
    const uint64_t dim = (uint64_t)1 << n;
#pragma omp parallel for schedule(static) if (dim >= ORC_PAR_MIN)
    for (uint64_t i = 0; i < dim; ++i) {
        uint64_t o = 0;
        for (int q = 0; q < n; ++q)
            if (i & ((uint64_t)1 << q)) o |= (uint64_t)1 << perm[q];
        out[o] = in[i];
    }
}

/* ------------------------------------------------------------------------- */
/* Reductions (plain FP64 sums in index order).                               */
/* ------------------------------------------------------------------------- */
double orc_norm2(const cplx *psi, int n)
{
    const uint64_t dim = (uint64_t)1 << n;
    double s = 0;
    for (uint64_t i = 0; i < dim; ++i) s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    return s;
}

/* <Z_q> = sum_i |a_i|^2 (1 - 2 bit_q(i)) for every q; out has n entries. */
void orc_expect_z(const cplx *psi, int n, double *out)
{
    const uint64_t dim = (uint64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1) if (dim >= ORC_PAR_MIN)
    for (int q = 0; q < n; ++q) {
        double s = 0;
        for (uint64_t i = 0; i < dim; ++i) {
            const double p = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
            s += ((i >> q) & 1) ? -p : p;
        }
        out[q] = s;
    }
}

/* <psi| P |psi> for the Pauli string P with X on the qubits of xmask only,   */
/* Z on zmask only and Y on both. P|i> = i^{#Y} (-1)^{popcount(i & zmask)}     */
/* |i XOR xmask> (Y|0> = i|1>, Y|1> = -i|0>). Returns the real part.          */
double orc_expect_pauli(const cplx *psi, int n, uint64_t xmask, uint64_t zmask)
{
    const uint64_t dim = (uint64_t)1 << n;
    int ny = 0;
    for (int q = 0; q < n; ++q)
        if (((xmask >> q) & 1) && ((zmask >> q) & 1)) ++ny;
    cplx iy = 1;
    for (int y = 0; y < ny; ++y) iy *= I;
    cplx s = 0;
    for (uint64_t i = 0; i < dim; ++i) {
        const int sign = __builtin_parityll(i & zmask);   /* (-1)^popcount */
        const cplx pi = iy * (sign ? -psi[i] : psi[i]);   /* component of P|psi> at i ^ xmask */
        s += conj(psi[i ^ xmask]) * pi;
    }
    return creal(s);
}

/* H|psi> for H = sum_t coeff[t] P_t (out must not alias psi). */
void orc_apply_pauli_sum(const cplx *psi, cplx *out, int n, const double *coeff,
                         const uint64_t *xmask, const uint64_t *zmask, int64_t nt)
{
    const uint64_t dim = (uint64_t)1 << n;
    for (uint64_t i = 0; i < dim; ++i) out[i] = 0;
    for (int64_t t = 0; t < nt; ++t) {
        int ny = 0;
        for (int q = 0; q < n; ++q)
            if (((xmask[t] >> q) & 1) && ((zmask[t] >> q) & 1)) ++ny;
        cplx iy = 1;
        for (int y = 0; y < ny; ++y) iy *= I;
        for (uint64_t i = 0; i < dim; ++i) {
            const int sign = __builtin_parityll(i & zmask[t]);
            out[i ^ xmask[t]] += coeff[t] * iy * (sign ? -psi[i] : psi[i]);
        }
    }
}

