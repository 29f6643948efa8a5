/*
 * vqe.h -- C ABI of the GB300 VQE hot-path library (libvqe_gb300.so).
 *
 * The library evaluates, on one GPU, the inner loop of the variational
 * quantum eigensolver of Morita, Tomita, Koyama, Kimura, "Simulator
 * Demonstration of Large Scale Variational Quantum Algorithm on HPC Cluster"
 * (2024):
 *   - a parameterised hardware-efficient ansatz applied to a 2^n-amplitude
 *     state vector (Sec. II-B, Eq. 6; the paper names this ansatz class),
 *   - the energy <psi|H|psi>/<psi|psi> of a qubit Hamiltonian given as a
 *     Pauli sum H = sum_i w_i P_i (Sec. II-B, Eqs. 2-4 and 7),
 *   - the Hamiltonian cutoff ("slimming"): terms with |w| below a threshold
 *     are dropped and the bound sum |w_dropped| is reported (Sec. II-D,
 *     Sec. III-D),
 *   - the gradient of the energy by adjoint differentiation (the paper
 *     instead spends one circuit evaluation per parameter, Sec. II-C).
 *
 * Conventions (all calls):
 *   - Qubit q is bit q of a basis-state index; |0...0> is index 0.
 *   - A Pauli string is a pair of bit masks (x, z): per qubit (0,0)=I,
 *     (1,0)=X, (0,1)=Z, (1,1)=Y.  The coefficient multiplies the tensor
 *     product of those matrices.
 *   - Ansatz: depth D layers; layer l applies, on every qubit q,
 *     RY(theta_{l,q}) = [[c,-s],[s,c]] (c = cos theta/2, s = sin theta/2)
 *     then RZ(phi_{l,q}) = diag(e^{-i phi/2}, e^{+i phi/2}), then CZ(q, q+1)
 *     for q = 0..n-2.  Parameter layout (2nD doubles):
 *     params[(l*n + q)*2] = theta_{l,q}, params[(l*n + q)*2 + 1] = phi_{l,q}.
 *     The circuit starts from |0...0>.
 *   - State layout: 2^n interleaved complex numbers (re, im): float2 in
 *     VQE_C64 mode, double2 in VQE_C128 mode; batched states are stored
 *     back to back.
 *   - Energies are <psi|H|psi>/<psi|psi> (Eq. 7); gradients are of the
 *     unnormalised <psi|H|psi> (equal for the unitary circuit).
 *   - Precision: VQE_C128 computes everything in FP64.  VQE_C64 keeps the
 *     state in complex64 and does gate arithmetic in FP32, and accumulates
 *     energies, norms and gradients in FP64.
 *
 * Ownership and threading: a handle is used by one host thread at a time.
 * Host arrays passed in are copied before the call returns.  Device pointers
 * passed in stay owned by the caller.  All device work is queued on the
 * stream given at creation; calls that return numbers to host memory
 * synchronise that stream before returning, the *_dev batch calls do not.
 *
 * Errors: every call returns a vqe_status; on error the handle's previous
 * Hamiltonian, state and workspace are left as they were, and
 * vqe_last_error() describes the failure.  A CUDA error inside a call is
 * returned as VQE_ERR_CUDA.
 */
#ifndef VQE_GB300_H
#define VQE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vqe_ctx *vqe_handle;

typedef enum {
    VQE_OK = 0,
    VQE_ERR_ARG = 1,      /* invalid argument (range, NULL, size, non-finite value) */
    VQE_ERR_STATE = 2,    /* call out of order (e.g. energy before any ansatz) */
    VQE_ERR_OOM = 3,      /* device memory could not be allocated */
    VQE_ERR_CUDA = 4,     /* a CUDA runtime call or kernel launch failed */
    VQE_ERR_TIMEOUT = 5,  /* reserved (no call of this version returns it) */
    VQE_ERR_DEVICE = 6    /* reserved (no call of this version returns it) */
} vqe_status;

typedef enum { VQE_C64 = 0, VQE_C128 = 1 } vqe_precision;

/* Per-handle counters, for reports and tests. */
typedef struct {
    uint64_t kernel_launches;   /* kernels this handle launched since creation (graph nodes count) */
    uint64_t n_terms_input;     /* terms passed to vqe_set_hamiltonian */
    uint64_t n_terms_canonical; /* after merging equal strings and removing zeros */
    uint64_t n_terms_kept;      /* after the last vqe_slim */
    uint64_t n_groups;          /* distinct x masks among kept terms */
    double   sum_abs_dropped;   /* bound of the last vqe_slim */
    double   threshold;         /* threshold of the last vqe_slim */
    uint32_t ansatz_passes;     /* tile passes per circuit evaluation */
    uint32_t tile_bits_max;     /* largest tile (log2 amplitudes) the pass plan uses */
} vqe_stats;

/* Create a handle for n_qubits (1..32) and depth (>= 1) layers.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  The device is
 * the one current on the calling thread. */
vqe_status vqe_create(int n_qubits, int depth, vqe_precision precision, void *cuda_stream,
                      vqe_handle *out);
/* Create a handle whose ansatz is the particle-conserving one of Sec. II-B
 * (Eqs. 5-6): psi(theta) = U(theta) psi_HF, psi_HF the basis state with modes
 * 0 .. n_elec-1 occupied (mode m = qubit m, occupied = 1, Jordan-Wigner
 * mapping), and U the product of n_exc fermionic excitation gates
 * exp(theta_j (T_j - T_j^dag)) applied in the order given.  Excitation j is
 * four ints excitations[4j .. 4j+3] = (p, q, r, s):
 *   q >= 0: double, T = a_p^dag a_q^dag a_r a_s (p, q, r, s distinct);
 *   q = -1 and s = -1: single, T = a_p^dag a_r (p != r).
 * Modes must lie in 0 .. n_qubits-1 (VQE_ERR_ARG otherwise).  Parameters are
 * theta_j, one per excitation (n_exc doubles).  Every other call works as for
 * vqe_create (Hamiltonian, cutoff, energies, adjoint gradients, batches,
 * autotuner) except vqe_set_plan_options and the one-gate-per-pass kernel,
 * which return VQE_ERR_ARG.  The array is copied.  Consecutive gates whose
 * modes fit one shared-memory tile share one pass over the state. */
vqe_status vqe_create_pc(int n_qubits, int n_elec, int n_exc, const int *excitations,
                         vqe_precision precision, void *cuda_stream, vqe_handle *out);

/* Free the handle and every device buffer the library allocated. */
vqe_status vqe_destroy(vqe_handle h);

/* Device bytes of state workspace for `batch` states, with (want_gradient=1)
 * or without the adjoint buffers. */
vqe_status vqe_workspace_size(vqe_handle h, int batch, int want_gradient, size_t *bytes);
/* Use caller-owned device memory (at least 256-byte aligned) as the state
 * workspace; the library never frees it.  Pass NULL to return to
 * library-allocated workspace.  The batch capacity follows from `bytes`. */
vqe_status vqe_bind_workspace(vqe_handle h, void *dev_ptr, size_t bytes);

/* Tile plan of the ansatz passes (0 = default for each): tile_bits_max =
 * log2 of the largest tile a pass stages in shared memory (1..14; default
 * 11), run_bits = log2 of the contiguous run of amplitudes at least kept in
 * the tiles of high-qubit passes (default 2 for C128, 3 for C64: 64 bytes),
 * reg_bits = log2 of the amplitudes each thread
 * holds (1..5; default 3 for C128, 4 for C64).  reg_bits 5 applies to energy
 * evaluations only; gradients use at most 4.
 * Rejected (VQE_ERR_ARG) if a pass would need more than 512 threads or
 * 227 KiB of shared memory.  Rebuilds the plans; the state of
 * vqe_apply_ansatz is discarded.  Results do not depend on the plan beyond
 * floating-point rounding order. */
vqe_status vqe_set_plan_options(vqe_handle h, int tile_bits_max, int run_bits, int reg_bits);

/* Form of lambda = H psi in gradient evaluations (the adjoint's apply-H):
 * mode 0 = one sweep over the state that gathers psi_{i^x} for every X-mask
 * group; mode 1 = accumulated window by window over the expectation's tile
 * windows (where every group fits a window); mode 2 = bit-ordered sweeps:
 * the groups are split into a few sweeps whose state order makes the X bits
 * of their groups run fastest, so that the gathered partners are read from
 * L2 (where every group's terms fit a sweep); a form the Hamiltonian cannot
 * use falls back to mode 0.  Mode -1 (default) = mode 2 when every group's
 * nonzero terms form one merged term on one parity of its X bits (hopping
 * Hamiltonians), else windows when they hold at least 10 groups each, else
 * mode 0; the autotuner times all three.  The
 * choice persists across vqe_set_hamiltonian and vqe_slim; *form (may be
 * NULL) reports the form (0, 1 or 2) the current Hamiltonian will use.
 * Results agree to rounding order.  VQE_ERR_ARG for a mode outside -1..2. */
vqe_status vqe_set_apply_mode(vqe_handle h, int mode, int *form);

/* Set the Hamiltonian H = sum_t coeffs[t] * P(x_masks[t], z_masks[t])
 * (Sec. II-B, Eqs. 2-4).  Host arrays of length n_terms; masks must have no
 * bit at or above n_qubits; coefficients must be finite.  Equal strings are
 * merged (coefficients summed) and exact zeros removed; the kept set is the
 * whole canonical Hamiltonian until vqe_slim is called. */
vqe_status vqe_set_hamiltonian(vqe_handle h, const uint64_t *x_masks, const uint64_t *z_masks,
                               const double *coeffs, size_t n_terms);

/* Hamiltonian cutoff (Sec. II-D and III-D): keep exactly the canonical
 * terms with |c| >= threshold (threshold 0 keeps all), report the kept count
 * and sum |c| over dropped terms, the bound on |E_full - E_slim| * <psi|psi>
 * (Sec. II-D).  Always starts again from the full canonical set.  Either
 * output pointer may be NULL. */
vqe_status vqe_slim(vqe_handle h, double threshold, size_t *n_kept, double *sum_abs_dropped);

/* Apply the ansatz with host parameters (2*n*depth doubles) to |0...0> and
 * keep the state in the handle (batch slot 0). */
vqe_status vqe_apply_ansatz(vqe_handle h, const double *params);

/* Energy <psi|H|psi>/<psi|psi> and <psi|psi> of the state left by the last
 * vqe_apply_ansatz (Eq. 7), with the kept terms.  Either pointer may be NULL. */
vqe_status vqe_energy(vqe_handle h, double *energy, double *norm);

/* Copy the state of batch slot 0 to host memory (bytes = 2^n * 8 for C64,
 * 2^n * 16 for C128). */
vqe_status vqe_get_state(vqe_handle h, void *host_out, size_t bytes);

/* Run the ansatz with host params, then return the adjoint gradient
 * d<psi|H|psi>/d params (2*n*depth doubles, host) and the energy.  The state
 * afterwards is undefined (the backward sweep consumes it). */
vqe_status vqe_gradient(vqe_handle h, const double *params, double *grad, double *energy);

/* Batched evaluation with device-resident buffers, queued on the handle's
 * stream without synchronising:
 *   params_dev:   batch * 2*n*depth doubles
 *   energies_dev: batch doubles (E = <H>/<psi|psi>), norms_dev: batch doubles or NULL
 *   grads_dev:    batch * 2*n*depth doubles (gradient call only)
 * Batches larger than the workspace capacity run in chunks. */
vqe_status vqe_energy_batch_dev(vqe_handle h, const double *params_dev, int batch,
                                double *energies_dev, double *norms_dev);
vqe_status vqe_gradient_batch_dev(vqe_handle h, const double *params_dev, int batch,
                                  double *grads_dev, double *energies_dev);

/* The same with host buffers (copies inside; synchronises). */
vqe_status vqe_energy_batch(vqe_handle h, const double *params, int batch, double *energies,
                            double *norms);
vqe_status vqe_gradient_batch(vqe_handle h, const double *params, int batch, double *grads,
                              double *energies);

/* Reference kernel for comparison: the same circuit with one gate per pass
 * over the state (RY, RZ and each CZ separately, as a per-gate simulator
 * does), then the same energy kernel.  Device buffers as above. */
vqe_status vqe_energy_batch_pergate_dev(vqe_handle h, const double *params_dev, int batch,
                                        double *energies_dev, double *norms_dev);

vqe_status vqe_get_stats(vqe_handle h, vqe_stats *out);

/* Autotuner: times the evaluation of `batch` parameter vectors (device
 * memory, as the *_batch_dev calls take them; gradient = 1 times energy +
 * adjoint gradient, 0 the energy) under candidate tile plans (the default
 * first, then other tile sizes -- the qubits fused per pass --, register
 * counts and run lengths; see vqe_set_plan_options), and, for gradients, the
 * possible forms of lambda = H psi (vqe_set_apply_mode) on the same state.  It keeps
 * the fastest plan and form on the handle.  Candidates after the default are
 * tried while the summed timed milliseconds stay below budget_ms.  Each
 * candidate runs once untimed (while evaluations take under 2 s) and once
 * timed with CUDA events on the handle's stream; the call synchronises.
 * Results of every candidate agree to rounding order.  The state of
 * vqe_apply_ansatz is discarded.  out (may be NULL) receives the choice. */
typedef struct {
    int tile_bits_max, run_bits, reg_bits;   /* chosen plan options (resolved values) */
    int apply_form;                          /* chosen form of lambda = H psi (vqe_set_apply_mode) */
    int candidates;                          /* plans timed */
    double ms_default, ms_best;              /* per evaluation: default plan, chosen plan */
    /* per state, gradient tuning only; 0 for a form not possible or not timed */
    double apply_ms_global, apply_ms_windows, apply_ms_sweeps;
} vqe_tuning;
vqe_status vqe_autotune(vqe_handle h, const double *params_dev, int batch, int gradient,
                        double budget_ms, vqe_tuning *out);

/* Kernel timing by CUDA events on the handle's stream.  When enabled, each
 * evaluation chunk records an event pair around each of its kernel groups:
 *   0 = forward ansatz passes, 1 = energy kernel, 2 = apply-H kernel,
 *   3 = backward (adjoint) passes.
 * ms[i] sums the elapsed times of group i; launches[i] counts the kernels
 * inside those intervals (back-to-back launches, so ms/launches is the mean
 * launch duration).  Enabling clears the counters; vqe_profile_read
 * synchronises the stream.  Event recording adds a few microseconds per
 * chunk. */
typedef struct {
    uint64_t launches[4];
    double ms[4];
    uint64_t chunks[4];
} vqe_kernel_times;
vqe_status vqe_profile(vqe_handle h, int enable);
vqe_status vqe_profile_read(vqe_handle h, vqe_kernel_times *out);

/* Message of the last failed call on this handle ("" if none).  The pointer
 * stays valid until the next call on the handle. */
const char *vqe_last_error(vqe_handle h);

/* Library version string. */
const char *vqe_version(void);

/* ---- Batched driver ------------------------------------------------------
 * Many independent problems of uneven size (the single-GPU counterpart of
 * the paper's distributed processing of independent circuit evaluations,
 * Sec. II-C): instance i has n_qubits[i] (1..24) qubits, depth[i] (1..64)
 * ansatz layers and its own Hamiltonian and parameters.  One run computes,
 * for every instance, the energy <psi|H|psi>/<psi|psi> and the adjoint
 * gradient, with persistent CTAs (each takes whole instances from a queue
 * ordered largest first; states that fit one tile stay in shared memory):
 * one kernel for the instances whose plans hold 16 amplitudes per thread,
 * one for the rest, both launched through ONE CUDA graph captured on first
 * use (vqe_batch_launch_count counts graph launches).
 *
 * Parameters and gradients of all instances are concatenated: instance i
 * owns entries [offsets[i], offsets[i+1]) (vqe_batch_param_offsets), laid
 * out as for vqe_create.  Every instance needs a Hamiltonian before a run
 * (VQE_ERR_STATE otherwise).  The library allocates device memory at
 * creation and on the first run: per-CTA scratch of 2 * 2^n amplitudes for
 * the largest instance that does not fit one tile.  cuda_stream NULL: the
 * batch uses an internal stream and vqe_batch_run_dev synchronises. */
typedef struct vqe_batch_ctx *vqe_batch;
vqe_status vqe_batch_create(int count, const int *n_qubits, const int *depths,
                            vqe_precision precision, void *cuda_stream, vqe_batch *out);
vqe_status vqe_batch_destroy(vqe_batch b);
vqe_status vqe_batch_set_hamiltonian(vqe_batch b, int instance, const uint64_t *x_masks,
                                     const uint64_t *z_masks, const double *coeffs,
                                     size_t n_terms);
/* offsets: count + 1 entries. */
vqe_status vqe_batch_param_offsets(vqe_batch b, size_t *offsets);
/* Device buffers: params and grads as the offsets say, energies[count]. */
vqe_status vqe_batch_run_dev(vqe_batch b, const double *params_dev, double *energies_dev,
                             double *grads_dev);
/* Host buffers (copies inside; synchronises). */
vqe_status vqe_batch_run(vqe_batch b, const double *params, double *energies, double *grads);
/* Tile size (log2 amplitudes, 10..13 for C64, 10..12 for C128) of the passes
 * of instances larger than one tile. */
vqe_status vqe_batch_set_tile_bits(vqe_batch b, int tile_bits);
/* Autotuner: times `reps` runs for each candidate tile size on the given
 * device buffers, keeps the fastest (reported in *tile_bits_out if not
 * NULL) and leaves the buffers holding a run with it. */
vqe_status vqe_batch_autotune(vqe_batch b, const double *params_dev, double *energies_dev,
                              double *grads_dev, int reps, int *tile_bits_out);
/* Graph launches so far (each launch runs one memset and one kernel). */
vqe_status vqe_batch_launch_count(vqe_batch b, uint64_t *graph_launches);
const char *vqe_batch_last_error(vqe_batch b);

/* ---- Energy without device allocation ------------------------------------
 * The paper has no counterpart of this call; it exists for users of this
 * library whose code may not allocate device memory: code whose device memory
 * is owned by another allocator (a framework's caching allocator or a fixed
 * pre-reserved pool), loops that keep other streams busy and cannot afford
 * the device-wide synchronisation of cudaMalloc/cudaFree, and plug-ins that
 * only receive raw device pointers from their host application.
 *
 * It computes, for `batch` states stored back to back at psi_dev (2^n
 * complex64 or complex128 each, as `precision` says), the energy
 * <psi|H|psi>/<psi|psi> of H = sum_t c_t P(x_t, z_t), taking the terms one at
 * a time (no merging, grouping or cutoff), and writes energies_dev[batch] and,
 * if not NULL, norms_dev[batch].  All arrays are caller-owned device memory;
 * the call itself allocates nothing.  Its only scratch is a fixed array of
 * 2 * VQE_NOALLOC_MAX_BATCH + 32 doubles (64 KiB) in the library's static
 * device memory, present on every GPU that loads the library until exit.
 *
 * Limits and errors: batch must be 1..VQE_NOALLOC_MAX_BATCH and n_qubits
 * 1..32, else VQE_ERR_ARG is returned before any work is queued.  Masks with
 * bits at or above n_qubits or non-finite coefficients cannot be checked on
 * the host (they are in device memory): such terms are skipped and every
 * energy of the call is set to NaN.
 *
 * The work is queued on cuda_stream (NULL = legacy default stream) and the
 * call returns without synchronising.  The first call on a device looks up
 * the scratch array's device address with that device current (the device
 * current on the calling thread); make that first call before any stream
 * capture.  Every call uses the same scratch array and overwrites what the
 * previous call left there; each slot a call reads is written by that call
 * first, so nothing needs clearing, but two calls that overlap on the GPU
 * (on different streams, or from different threads) race on the scratch and
 * give wrong results: serialise them. */
#define VQE_NOALLOC_MAX_BATCH 4096
vqe_status vqe_energy_noalloc(int n_qubits, vqe_precision precision, const void *psi_dev,
                              int batch, const uint64_t *x_masks_dev, const uint64_t *z_masks_dev,
                              const double *coeffs_dev, size_t n_terms, double *energies_dev,
                              double *norms_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
