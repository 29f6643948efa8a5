/*
 * Plain FP64 CPU oracle for the VQE hot path of "Simulator Demonstration of
 * Large Scale Variational Quantum Algorithm on HPC Cluster" (Morita et al.).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  The CUDA library never
 * links, calls or includes it, and it includes nothing from the CUDA side.
 *
 * State vectors are arrays of 2^n `double complex` (interleaved re, im);
 * qubit q is bit q of the basis index.  Pauli strings are bit masks (x, z):
 * per qubit (0,0)=I, (1,0)=X, (0,1)=Z, (1,1)=Y (Sec. II-B, Eqs. 2-4).
 *
 * Ansatz (hardware-efficient, Sec. II-B names the class): per layer l, for
 * each qubit q in order, RY(theta_{l,q}) then RZ(phi_{l,q}); then CZ(q, q+1)
 * for q = 0..n-2.  params[(l*n+q)*2] = theta, params[(l*n+q)*2+1] = phi.
 * RY(t) = [[cos t/2, -sin t/2], [sin t/2, cos t/2]],
 * RZ(p) = diag(exp(-i p/2), exp(+i p/2)).
 */
#ifndef VQE_ORACLE_H
#define VQE_ORACLE_H

#include <complex.h>
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* 2x2 gate u (row major) on qubit q. */
void orc_apply_1q(int n, double complex *psi, int q, const double complex u[4]);
void orc_ry_matrix(double theta, double complex u[4]);
void orc_rz_matrix(double phi, double complex u[4]);
void orc_apply_cz(int n, double complex *psi, int a, int b);

/* psi <- U(params) |0...0>  (Eq. 6 with |0...0> as the reference state). */
void orc_ansatz(int n, int depth, const double *params, double complex *psi);

/* out <- P(x, z) psi, each qubit's Pauli matrix applied explicitly. */
void orc_pauli_apply(int n, const double complex *psi, uint64_t x, uint64_t z,
                     double complex *out);

/* <psi|H|psi> (unnormalised; real and imaginary part) and <psi|psi>. */
void orc_expectation(int n, const double complex *psi, size_t n_terms,
                     const uint64_t *x, const uint64_t *z, const double *c,
                     double *e_re, double *e_im, double *norm);

/* lambda <- H psi. */
void orc_apply_h(int n, const double complex *psi, size_t n_terms,
                 const uint64_t *x, const uint64_t *z, const double *c,
                 double complex *lambda);

/* Canonical form: equal (x, z) merged by summing coefficients, exact zeros
 * removed, then every term with |c| < threshold dropped (Sec. II-D).  Output
 * arrays need room for n_terms entries, sorted by (x, z).  Returns the kept
 * count; *sum_abs_dropped receives the sum of |c| over dropped merged terms. */
size_t orc_slim(size_t n_terms, const uint64_t *x, const uint64_t *z, const double *c,
                double threshold, uint64_t *x_out, uint64_t *z_out, double *c_out,
                double *sum_abs_dropped);

/* Gradients of the unnormalised energy <psi(params)|H|psi(params)>:
 * adjoint differentiation, parameter shift (+-pi/2), central differences. */
void orc_gradient_adjoint(int n, int depth, const double *params, size_t n_terms,
                          const uint64_t *x, const uint64_t *z, const double *c,
                          double *grad, double *energy);
void orc_gradient_shift(int n, int depth, const double *params, size_t n_terms,
                        const uint64_t *x, const uint64_t *z, const double *c,
                        double *grad);
void orc_gradient_fd(int n, int depth, const double *params, size_t n_terms,
                     const uint64_t *x, const uint64_t *z, const double *c,
                     double h, double *grad);

/* Particle-conserving ansatz (Sec. II-B, Eqs. 5-6): excitation k is four
 * ints exc[4k..4k+3] = (p, q, r, s), the operator T = a_p^dag a_q^dag a_r a_s
 * (double) or, with q = -1, T = a_p^dag a_r (single; s ignored); its gate is
 * exp(theta_k (T - T^dag)) under the Jordan-Wigner mapping.  The circuit
 * applies excitations 0, 1, ... in order to psi_HF = the basis state with
 * modes 0 .. n_elec-1 occupied. */
void orc_apply_excitation(int n, double complex *psi, const int exc[4], double theta);
/* out <- (T - T^dag) psi */
void orc_excitation_generator(int n, const double complex *psi, const int exc[4],
                              double complex *out);
void orc_pc_ansatz(int n, int n_elec, int n_exc, const int *exc, const double *theta,
                   double complex *psi);
void orc_pc_gradient_adjoint(int n, int n_elec, int n_exc, const int *exc, const double *theta,
                             size_t n_terms, const uint64_t *x, const uint64_t *z,
                             const double *c, double *grad, double *energy);
void orc_pc_gradient_fd(int n, int n_elec, int n_exc, const int *exc, const double *theta,
                        size_t n_terms, const uint64_t *x, const uint64_t *z, const double *c,
                        double h, double *grad);

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
