/*
 * vqe_inspect.h -- host-only inspection of the plans libvqe_gb300 builds.
 *
 * These calls run the library's own planners on the host and copy their
 * output out, without touching a GPU, so tests can check the plans' index
 * arithmetic and semantics on a machine with no GPU.  The record layouts
 * are the library's internal structures; vqe_inspect_sizeof() reports their
 * sizes so a caller can verify that it mirrors them correctly.
 */
#ifndef VQE_GB300_INSPECT_H
#define VQE_GB300_INSPECT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* sizeof of internal record `which`: 0 = pass descriptor, 1 = staging slot,
 * 2 = term group, 3 = energy window, 4 = window group, 5 = window term,
 * 6 = excitation pass, 7 = excitation gate, 8 = apply-H sweep, 9 = sweep
 * group; 0 for an unknown `which`. */
size_t vqe_inspect_sizeof(int which);

/* Tile-pass plan of the ansatz for (n, depth, precision, options) -- options
 * as vqe_set_plan_options (tile_bits_max, run_bits, reg_bits; NULL = defaults):
 * forward and
 * backward pass descriptors (max_passes each), staging slots (max_stage),
 * and the gradient reduction map grad_map[3 * 2*n*depth] = (offset, count,
 * step) per parameter.  strides[3] = per-state coefficient, table and
 * gradient-partial sizes; counts[3] = passes, staging slots, parameters.
 * Returns 0, or -1 on invalid arguments or too-small buffers. */
int vqe_inspect_plan(int n_qubits, int depth, int precision, const int options[3], void *fwd,
                     void *bwd, int max_passes, void *stage, int max_stage, int *grad_map,
                     int max_params, uint64_t strides[3], int counts[3]);

/* Canonicalisation, cutoff and X-mask grouping of a Pauli sum, exactly as
 * vqe_set_hamiltonian followed by vqe_slim(threshold) prepare it: term
 * groups (max_groups), per-term z masks and sign-folded coefficients
 * (max_terms).  counts[2] = groups, terms; *sum_abs_dropped and
 * *n_canonical as vqe_slim and vqe_get_stats report them.  Returns 0, or -1
 * on invalid input (masks beyond n_qubits, non-finite values) or
 * too-small buffers. */
int vqe_inspect_hamiltonian(int n_qubits, const uint64_t *x_masks, const uint64_t *z_masks,
                            const double *coeffs, size_t n_terms, double threshold, void *groups,
                            int max_groups, uint32_t *tz, double *tc, int max_terms, int counts[2],
                            double *sum_abs_dropped, uint64_t *n_canonical);

/* Windows of the windowed expectation kernel for the same prepared terms
 * (Sec. II-B Eq. 7 evaluated per X-mask group): window records
 * (max_windows), window groups with their register-pattern runs
 * (max_wgroups), window terms (tile-coordinate Z bits, tile-number Z bits,
 * coefficient; max_wterms), the windows' high-part offset tables (max_hoff),
 * and the groups swept over the whole state instead (max_wide).  diag_terms:
 * 1 = keep the diagonal group's terms in the low window, 0 = leave them out
 * (the library does so when it precomputes the diagonal of H).
 * The windowed apply-H of the adjoint uses the same windows.
 * counts[5] = windows, window groups, window terms, offsets, wide groups.
 * Returns 0, or -1 on invalid input or too-small buffers. */
int vqe_inspect_windows(int n_qubits, int precision, const uint64_t *x_masks,
                        const uint64_t *z_masks, const double *coeffs, size_t n_terms,
                        double threshold, int diag_terms, void *windows,
                        int max_windows,
                        void *wgroups, int max_wgroups, void *wterms, int max_wterms,
                        uint32_t *hoff, int max_hoff, void *wide, int max_wide, int counts[5]);

/* Sweeps of the sweep form of lambda = H psi (vqe_set_apply_mode 2) for the
 * same prepared terms: sweep records (max_sweeps), sweep groups
 * (max_groups), pattern entries (first term | count << 16, max_pat), merged terms (Z bits and
 * A / B coefficients, max_terms), and the sweeps' bit-order tables (1024
 * entries per sweep: counter byte b with value v maps to order[1024 * w +
 * 256 * b + v]).  diag_terms as for vqe_inspect_windows.  counts[4] =
 * sweeps, groups, pattern entries, terms.  Returns 0, or -1 on invalid
 * input, too-small buffers, or a Hamiltonian whose groups do not fit the
 * sweeps (the library then uses another form). */
int vqe_inspect_sweeps(int n_qubits, int precision, const uint64_t *x_masks,
                       const uint64_t *z_masks, const double *coeffs, size_t n_terms,
                       double threshold, int diag_terms, void *sweeps, int max_sweeps,
                       void *groups, int max_groups, uint32_t *pat, int max_pat, uint32_t *tz,
                       double *ta, double *tb, int max_terms, uint32_t *order, int max_order,
                       int counts[4]);

/* Pass plan of the particle-conserving ansatz (vqe_create_pc) for the same
 * arguments: excitation passes (max_passes) with their support masks, their
 * gates with tile masks and sign masks (max_gates), and the passes'
 * high-part offset tables (max_hoff).  counts[3] = passes, gates, offsets.
 * Returns 0, or -1 on invalid arguments or too-small buffers. */
int vqe_inspect_pc_plan(int n_qubits, int n_elec, int precision, int n_exc, const int *excitations,
                        void *passes, int max_passes, void *gates, int max_gates, uint32_t *hoff,
                        int max_hoff, int counts[3]);

#ifdef __cplusplus
}
#endif
#endif
