/*
 * Plain FP64 CPU oracle: the definitions of the VQE hot path written out
 * one gate and one Pauli term at a time.  TEST INFRASTRUCTURE (see header).
 *
 * Everything here follows the textbook definitions the paper relies on:
 *   - psi(theta) = U(theta) psi_0                       (Sec. II-B, Eq. 6)
 *   - E = <psi|H|psi> / <psi|psi>, H = sum_i w_i P_i     (Eqs. 2-4 and 7)
 *   - cutoff: drop terms with |w| below Th_1            (Sec. II-D / III-D)
 *   - gradient: adjoint differentiation, checked against the parameter
 *     shift rule and central differences.
 * No blocking, fusion or reordering beyond those definitions.
 */
#include "vqe_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- gates */

void orc_ry_matrix(double theta, double complex u[4]) {
    double c = cos(theta / 2.0), s = sin(theta / 2.0);
    u[0] = c;  u[1] = -s;
    u[2] = s;  u[3] = c;
}

void orc_rz_matrix(double phi, double complex u[4]) {
    u[0] = cexp(-I * phi / 2.0);  u[1] = 0.0;
    u[2] = 0.0;                   u[3] = cexp(I * phi / 2.0);
}

void orc_apply_1q(int n, double complex *psi, int q, const double complex u[4]) {
    const int64_t dim = (int64_t)1 << n;
    const int64_t bit = (int64_t)1 << q;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; ++i) {
        if (i & bit) continue;               /* visit each pair (i, i|bit) once */
        int64_t j = i | bit;
        double complex a0 = psi[i], a1 = psi[j];
        psi[i] = u[0] * a0 + u[1] * a1;
        psi[j] = u[2] * a0 + u[3] * a1;
    }
}

void orc_apply_cz(int n, double complex *psi, int a, int b) {
    const int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; ++i) {
        if (((i >> a) & 1) && ((i >> b) & 1)) psi[i] = -psi[i];
    }
}

/* One entry of the gate sequence of the hardware-efficient ansatz. */
typedef struct { int kind; int q; int q2; int param; } orc_gate; /* kind 0 RY, 1 RZ, 2 CZ */

static int build_sequence(int n, int depth, orc_gate *seq) {
    int k = 0;
    for (int l = 0; l < depth; ++l) {
        for (int q = 0; q < n; ++q) {
            seq[k++] = (orc_gate){0, q, -1, (l * n + q) * 2 + 0};
            seq[k++] = (orc_gate){1, q, -1, (l * n + q) * 2 + 1};
        }
        for (int q = 0; q + 1 < n; ++q) seq[k++] = (orc_gate){2, q, q + 1, -1};
    }
    return k;
}

static void gate_matrix(const orc_gate *g, const double *params, double complex u[4]) {
    if (g->kind == 0) orc_ry_matrix(params[g->param], u);
    else orc_rz_matrix(params[g->param], u);
}

static void apply_gate(int n, double complex *psi, const orc_gate *g, const double *params,
                       int adjoint) {
    if (g->kind == 2) { orc_apply_cz(n, psi, g->q, g->q2); return; }
    double complex u[4];
    gate_matrix(g, params, u);
    if (adjoint) {
        double complex v[4] = {conj(u[0]), conj(u[2]), conj(u[1]), conj(u[3])};
        orc_apply_1q(n, psi, g->q, v);
    } else {
        orc_apply_1q(n, psi, g->q, u);
    }
}

void orc_ansatz(int n, int depth, const double *params, double complex *psi) {
    const int64_t dim = (int64_t)1 << n;
    memset(psi, 0, sizeof(double complex) * (size_t)dim);
    psi[0] = 1.0;
    int max_gates = depth * (3 * n);
    orc_gate *seq = (orc_gate *)malloc(sizeof(orc_gate) * (size_t)(max_gates + 1));
    int ng = build_sequence(n, depth, seq);
    for (int k = 0; k < ng; ++k) apply_gate(n, psi, &seq[k], params, 0);
    free(seq);
}

/* ---------------------------------------------------------------- Pauli */

/* P(x,z)|j> = phase(j) |j ^ x>, built qubit by qubit from
 * I|b> = |b>, X|b> = |1-b>, Z|b> = (-1)^b |b>, Y|0> = i|1>, Y|1> = -i|0>. */
static double complex pauli_phase(int n, uint64_t j, uint64_t x, uint64_t z) {
    double complex ph = 1.0;
    for (int k = 0; k < n; ++k) {
        int xb = (int)((x >> k) & 1), zb = (int)((z >> k) & 1), b = (int)((j >> k) & 1);
        if (!xb && !zb) continue;                 /* I */
        if (xb && !zb) continue;                  /* X: flips the bit, factor 1 */
        if (!xb && zb) { if (b) ph = -ph; continue; }   /* Z */
        ph *= b ? -I : I;                         /* Y */
    }
    return ph;
}

void orc_pauli_apply(int n, const double complex *psi, uint64_t x, uint64_t z,
                     double complex *out) {
    const int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < dim; ++j) {
        out[(uint64_t)j ^ x] = pauli_phase(n, (uint64_t)j, x, z) * psi[j];
    }
}

void orc_expectation(int n, const double complex *psi, size_t n_terms,
                     const uint64_t *x, const uint64_t *z, const double *c,
                     double *e_re, double *e_im, double *norm) {
    const int64_t dim = (int64_t)1 << n;
    double complex *tmp = (double complex *)malloc(sizeof(double complex) * (size_t)dim);
    double er = 0.0, ei = 0.0, nn = 0.0;
    for (int64_t i = 0; i < dim; ++i) nn += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    for (size_t t = 0; t < n_terms; ++t) {
        orc_pauli_apply(n, psi, x[t], z[t], tmp);
        double sr = 0.0, si = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sr, si)
        for (int64_t i = 0; i < dim; ++i) {
            double complex v = conj(psi[i]) * tmp[i];
            sr += creal(v);
            si += cimag(v);
        }
        er += c[t] * sr;
        ei += c[t] * si;
    }
    free(tmp);
    *e_re = er;
    *e_im = ei;
    *norm = nn;
}

void orc_apply_h(int n, const double complex *psi, size_t n_terms,
                 const uint64_t *x, const uint64_t *z, const double *c,
                 double complex *lambda) {
    const int64_t dim = (int64_t)1 << n;
    double complex *tmp = (double complex *)malloc(sizeof(double complex) * (size_t)dim);
    memset(lambda, 0, sizeof(double complex) * (size_t)dim);
    for (size_t t = 0; t < n_terms; ++t) {
        orc_pauli_apply(n, psi, x[t], z[t], tmp);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < dim; ++i) lambda[i] += c[t] * tmp[i];
    }
    free(tmp);
}

/* ---------------------------------------------------------------- cutoff */

typedef struct { uint64_t x, z; double c; } orc_term;

static int term_cmp(const void *a, const void *b) {
    const orc_term *p = (const orc_term *)a, *q = (const orc_term *)b;
    if (p->x != q->x) return p->x < q->x ? -1 : 1;
    if (p->z != q->z) return p->z < q->z ? -1 : 1;
    return 0;
}

size_t orc_slim(size_t n_terms, const uint64_t *x, const uint64_t *z, const double *c,
                double threshold, uint64_t *x_out, uint64_t *z_out, double *c_out,
                double *sum_abs_dropped) {
    orc_term *t = (orc_term *)malloc(sizeof(orc_term) * (n_terms ? n_terms : 1));
    for (size_t k = 0; k < n_terms; ++k) t[k] = (orc_term){x[k], z[k], c[k]};
    qsort(t, n_terms, sizeof(orc_term), term_cmp);
    size_t kept = 0;
    double dropped = 0.0;
    size_t k = 0;
    while (k < n_terms) {
        size_t e = k;
        double s = 0.0;
        while (e < n_terms && t[e].x == t[k].x && t[e].z == t[k].z) s += t[e++].c;
        if (s != 0.0) {
            if (fabs(s) < threshold) {
                dropped += fabs(s);
            } else {
                x_out[kept] = t[k].x;
                z_out[kept] = t[k].z;
                c_out[kept] = s;
                ++kept;
            }
        }
        k = e;
    }
    free(t);
    *sum_abs_dropped = dropped;
    return kept;
}

/* ---------------------------------------------------------------- gradient */

static double energy_of(int n, const double complex *psi, size_t T, const uint64_t *x,
                        const uint64_t *z, const double *c) {
    double er, ei, nn;
    orc_expectation(n, psi, T, x, z, c, &er, &ei, &nn);
    return er;
}

static void dgate_matrix(const orc_gate *g, const double *params, double complex d[4]) {
    double a = params[g->param];
    if (g->kind == 0) {       /* d/dt [[c,-s],[s,c]], c = cos t/2, s = sin t/2 */
        double c = cos(a / 2.0), s = sin(a / 2.0);
        d[0] = -s / 2.0;  d[1] = -c / 2.0;
        d[2] = c / 2.0;   d[3] = -s / 2.0;
    } else {                  /* d/dp diag(e^{-ip/2}, e^{ip/2}) */
        d[0] = -I / 2.0 * cexp(-I * a / 2.0);  d[1] = 0.0;
        d[2] = 0.0;                            d[3] = I / 2.0 * cexp(I * a / 2.0);
    }
}

void orc_gradient_adjoint(int n, int depth, const double *params, size_t n_terms,
                          const uint64_t *x, const uint64_t *z, const double *c,
                          double *grad, double *energy) {
    const int64_t dim = (int64_t)1 << n;
    const size_t bytes = sizeof(double complex) * (size_t)dim;
    double complex *psi = (double complex *)malloc(bytes);
    double complex *lam = (double complex *)malloc(bytes);
    double complex *mu = (double complex *)malloc(bytes);
    orc_gate *seq = (orc_gate *)malloc(sizeof(orc_gate) * (size_t)(depth * 3 * n + 1));
    int ng = build_sequence(n, depth, seq);

    orc_ansatz(n, depth, params, psi);
    orc_apply_h(n, psi, n_terms, x, z, c, lam);
    double e = 0.0;
    for (int64_t i = 0; i < dim; ++i) e += creal(conj(psi[i]) * lam[i]);
    *energy = e;

    /* Walk the gates backwards: psi <- U_k^dag psi (state before gate k),
     * g_k = 2 Re <lambda | dU_k | psi>, lambda <- U_k^dag lambda. */
    for (int k = ng - 1; k >= 0; --k) {
        const orc_gate *g = &seq[k];
        apply_gate(n, psi, g, params, 1);
        if (g->kind != 2) {
            double complex d[4];
            dgate_matrix(g, params, d);
            memcpy(mu, psi, bytes);
            orc_apply_1q(n, mu, g->q, d);
            double s = 0.0;
            for (int64_t i = 0; i < dim; ++i) s += creal(conj(lam[i]) * mu[i]);
            grad[g->param] = 2.0 * s;
        }
        apply_gate(n, lam, g, params, 1);
    }
    free(seq);
    free(mu);
    free(lam);
    free(psi);
}

void orc_gradient_shift(int n, int depth, const double *params, size_t n_terms,
                        const uint64_t *x, const uint64_t *z, const double *c,
                        double *grad) {
    const int np = 2 * n * depth;
    const int64_t dim = (int64_t)1 << n;
    double *p = (double *)malloc(sizeof(double) * (size_t)np);
    double complex *psi = (double complex *)malloc(sizeof(double complex) * (size_t)dim);
    for (int j = 0; j < np; ++j) {
        memcpy(p, params, sizeof(double) * (size_t)np);
        p[j] = params[j] + M_PI / 2.0;
        orc_ansatz(n, depth, p, psi);
        double ep = energy_of(n, psi, n_terms, x, z, c);
        p[j] = params[j] - M_PI / 2.0;
        orc_ansatz(n, depth, p, psi);
        double em = energy_of(n, psi, n_terms, x, z, c);
        grad[j] = (ep - em) / 2.0;
    }
    free(psi);
    free(p);
}

void orc_gradient_fd(int n, int depth, const double *params, size_t n_terms,
                     const uint64_t *x, const uint64_t *z, const double *c,
                     double h, double *grad) {
    const int np = 2 * n * depth;
    const int64_t dim = (int64_t)1 << n;
    double *p = (double *)malloc(sizeof(double) * (size_t)np);
    double complex *psi = (double complex *)malloc(sizeof(double complex) * (size_t)dim);
    for (int j = 0; j < np; ++j) {
        memcpy(p, params, sizeof(double) * (size_t)np);
        p[j] = params[j] + h;
        orc_ansatz(n, depth, p, psi);
        double ep = energy_of(n, psi, n_terms, x, z, c);
        p[j] = params[j] - h;
        orc_ansatz(n, depth, p, psi);
        double em = energy_of(n, psi, n_terms, x, z, c);
        grad[j] = (ep - em) / (2.0 * h);
    }
    free(psi);
    free(p);
}

/* ---------------------------------------------------------------- particle-conserving ansatz
 *
 * Sec. II-B, Eq. 5: U(theta) = prod D_pqrs(theta_pqrs) prod S_pq(theta_pq), applied to
 * the Hartree-Fock state (Eq. 6 with psi_HF).  The paper takes S and D from
 * an earlier gate set without printing them; the reading used here is the
 * fermionic excitation exp(theta (T - T^dag)) of the excitation operator
 * T = a_p^dag a_r (single) or T = a_p^dag a_q^dag a_r a_s (double) under the
 * Jordan-Wigner mapping (occupied mode m = bit m set), written out by
 * applying the ladder operators to basis states one at a time. */

/* a_m^dag (create = 1) or a_m (create = 0) on basis state *j: returns the
 * Jordan-Wigner sign (-1)^(number of occupied modes below m) and updates *j,
 * or returns 0 when the state is annihilated. */
static int jw_ladder(uint64_t *j, int m, int create) {
    const uint64_t bit = (uint64_t)1 << m;
    const int occupied = (*j & bit) != 0;
    if (create == occupied) return 0;
    int parity = 0;
    for (int k = 0; k < m; ++k) parity ^= (int)((*j >> k) & 1);
    *j ^= bit;
    return parity ? -1 : 1;
}

/* T|j> = sign |*out> for the excitation exc = (p, q, r, s): T = a_p^dag a_r
 * when q < 0 (s ignored), else a_p^dag a_q^dag a_r a_s; operators act right
 * to left.  Returns 0 when T|j> = 0. */
static int excitation_apply(const int exc[4], uint64_t j, uint64_t *out) {
    int sign = 1;
    if (exc[1] < 0) {
        int s1 = jw_ladder(&j, exc[2], 0);
        if (!s1) return 0;
        int s2 = jw_ladder(&j, exc[0], 1);
        if (!s2) return 0;
        sign = s1 * s2;
    } else {
        const int modes[4] = {exc[3], exc[2], exc[1], exc[0]};
        const int create[4] = {0, 0, 1, 1};
        for (int k = 0; k < 4; ++k) {
            int sk = jw_ladder(&j, modes[k], create[k]);
            if (!sk) return 0;
            sign *= sk;
        }
    }
    *out = j;
    return sign;
}

void orc_apply_excitation(int n, double complex *psi, const int exc[4], double theta) {
    const int64_t dim = (int64_t)1 << n;
    const double c = cos(theta), s = sin(theta);
    /* exp(theta G), G = T - T^dag, on each pair (j, j') with T|j> = sgn |j'>:
     * G|j> = sgn |j'>, G|j'> = -sgn |j>. */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < dim; ++j) {
        uint64_t jp;
        const int sgn = excitation_apply(exc, (uint64_t)j, &jp);
        if (!sgn) continue;
        const double complex a = psi[j], b = psi[jp];
        psi[j] = c * a - sgn * s * b;
        psi[jp] = c * b + sgn * s * a;
    }
}

void orc_excitation_generator(int n, const double complex *psi, const int exc[4],
                              double complex *out) {
    const int64_t dim = (int64_t)1 << n;
    memset(out, 0, sizeof(double complex) * (size_t)dim);
    for (int64_t j = 0; j < dim; ++j) {
        uint64_t jp;
        const int sgn = excitation_apply(exc, (uint64_t)j, &jp);
        if (!sgn) continue;
        out[jp] += sgn * psi[j];      /* T   |j>  = sgn |j'> */
        out[j] -= sgn * psi[jp];      /* -T^dag |j'> = -sgn |j> */
    }
}

void orc_pc_ansatz(int n, int n_elec, int n_exc, const int *exc, const double *theta,
                   double complex *psi) {
    const int64_t dim = (int64_t)1 << n;
    memset(psi, 0, sizeof(double complex) * (size_t)dim);
    const uint64_t hf = n_elec >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << n_elec) - 1);
    psi[hf] = 1.0;
    for (int k = 0; k < n_exc; ++k) orc_apply_excitation(n, psi, exc + 4 * k, theta[k]);
}

void orc_pc_gradient_adjoint(int n, int n_elec, int n_exc, const int *exc, const double *theta,
                             size_t n_terms, const uint64_t *x, const uint64_t *z,
                             const double *c, double *grad, double *energy) {
    const int64_t dim = (int64_t)1 << n;
    const size_t bytes = sizeof(double complex) * (size_t)dim;
    double complex *psi = (double complex *)malloc(bytes);
    double complex *lam = (double complex *)malloc(bytes);
    double complex *mu = (double complex *)malloc(bytes);
    orc_pc_ansatz(n, n_elec, n_exc, exc, theta, psi);
    orc_apply_h(n, psi, n_terms, x, z, c, lam);
    double e = 0.0;
    for (int64_t i = 0; i < dim; ++i) e += creal(conj(psi[i]) * lam[i]);
    *energy = e;
    /* psi holds U_k ... U_1 psi_HF and lambda the adjoint state at the same
     * point: g_k = 2 Re <lambda| G_k |psi>, then both step back through U_k. */
    for (int k = n_exc - 1; k >= 0; --k) {
        orc_excitation_generator(n, psi, exc + 4 * k, mu);
        double s = 0.0;
        for (int64_t i = 0; i < dim; ++i) s += creal(conj(lam[i]) * mu[i]);
        grad[k] = 2.0 * s;
        orc_apply_excitation(n, psi, exc + 4 * k, -theta[k]);
        orc_apply_excitation(n, lam, exc + 4 * k, -theta[k]);
    }
    free(mu);
    free(lam);
    free(psi);
}

void orc_pc_gradient_fd(int n, int n_elec, int n_exc, const int *exc, const double *theta,
                        size_t n_terms, const uint64_t *x, const uint64_t *z, const double *c,
                        double h, double *grad) {
    const int64_t dim = (int64_t)1 << n;
    double *p = (double *)malloc(sizeof(double) * (size_t)(n_exc ? n_exc : 1));
    double complex *psi = (double complex *)malloc(sizeof(double complex) * (size_t)dim);
    for (int j = 0; j < n_exc; ++j) {
        memcpy(p, theta, sizeof(double) * (size_t)n_exc);
        p[j] = theta[j] + h;
        orc_pc_ansatz(n, n_elec, n_exc, exc, p, psi);
        const double ep = energy_of(n, psi, n_terms, x, z, c);
        p[j] = theta[j] - h;
        orc_pc_ansatz(n, n_elec, n_exc, exc, p, psi);
        const double em = energy_of(n, psi, n_terms, x, z, c);
        grad[j] = (ep - em) / (2.0 * h);
    }
    free(psi);
    free(p);
}
