// Internal declarations shared by the host planner and the CUDA kernels of
// libvqe_gb300.  Nothing here is part of the public C ABI (include/vqe.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace vqe {

// ---------------------------------------------------------------- ansatz passes
//
// The ansatz layer l is  CZ_chain * prod_q RZ_q(phi_{l,q}) * prod_q RY_q(theta_{l,q}).
// Its qubits are split into groups; one "pass" stages one tile of 2^k
// amplitudes per CTA in shared memory, where the tile spans the pass's
// qubit group, and applies every gate of one or more layers that acts on
// those qubits.  A pass program is a list of ops interpreted by the kernel:
//   OP_ROUND(chunk)   move the thread's registers to a new set of R tile bits
//                     [chunk, chunk+R) (through shared memory; the first
//                     round loads from global memory)
//   OP_BF(slot,mask)  RY butterflies of `slot` on register bits in `mask`
//   OP_DIAG(slot)     RZ phases + RY scale (table) and CZ signs of `slot`
//   OP_FLUSH(slot)    (backward only) reduce this slot's gradient partials
// A "slot" is one layer's share of the pass.

constexpr int kMaxOps = 384;
constexpr int kMaxSlots = 40;
constexpr int kMaxTileBits = 14;

enum OpKind : uint8_t { OP_ROUND = 0, OP_BF = 1, OP_DIAG = 2, OP_FLUSH = 3 };

struct PassOp {
    uint8_t kind;
    uint8_t chunk;  // OP_ROUND: first tile bit of the register chunk
    uint8_t mask;   // OP_BF: register bits whose gate is applied
    uint8_t slot;   // OP_BF / OP_DIAG / OP_FLUSH: slot index within the pass
};

struct PassDesc {
    int k;          // tile bits (tile = 2^k amplitudes)
    int m;          // low tile bits = global bits [0, m) (contiguous run of 2^m amplitudes)
    int a;          // tile bits [m, k) = global bits [a, a + k - m)
    int R;          // register bits per thread (thread holds 2^R amplitudes)
    int n_ops;
    int n_slots;
    // Forward passes start from |0...0>: before this pass only the qubits
    // rotated by earlier passes can be 1, so a tile whose base has a bit of
    // zmask set is zero and stays zero.  Backward pass p carries the forward
    // zmask of pass p + 1: its tiles with a bit of it set hold psi = 0 and a
    // lambda no later gradient reads, and are skipped (zero partials).
    uint32_t zmask;
    int slot_layer[kMaxSlots];
    uint32_t slot_czmask[kMaxSlots];  // bit q: CZ(q, q+1) applied in this slot's DIAG
    uint32_t slot_gated[kMaxSlots];   // tile bits gated (RY, RZ) in this slot
    int slot_coef_off[kMaxSlots];     // per-state index of this slot's coefficient row (k entries)
    int slot_dtab_off[kMaxSlots];     // per-state index (complex entries) of this slot's 2^k table
    int slot_grad_off[kMaxSlots];     // per-state index (doubles) of this slot's gradient partials
    PassOp ops[kMaxOps];
};

// Rotation coefficient of one gated tile bit: RY(theta) = scale * B with
//   mode 0 ("tan"): B = [[1, -v], [v, 1]], v = tan(theta/2), scale = cos(theta/2)
//   mode 1 ("cot"): B = [[v, -1], [1, v]], v = cot(theta/2), scale = sin(theta/2)
// The mode keeps |v| <= 1.  The scales of a slot go into its diagonal table.
// In the backward sweep both buffers carry, when bit j's gradient is taken,
// the factor f_j = sigma / prod(scales of the bits un-rotated before j);
// gs = 1 / f_j^2 undoes it in the gradient partials.
template <typename T>
struct RotCoef {
    T v;
    T gs;
    int mode;
};

// Elements of one shared-memory tile buffer of 2^k amplitudes of elem_bytes
// each, including the padding of the layout between register rounds (one
// pad element per 128-byte row).
inline __host__ __device__ constexpr uint32_t tile_buf_elems(int k, int elem_bytes) {
    return (1u << k) + ((1u << k) >> (elem_bytes == 16 ? 3 : 4));
}

// Staging job: one slot of one pass (one row of coefficients and one table).
struct StageSlot {
    int k;             // tile bits of the pass
    int layer;
    int coef_off;      // per state
    int dtab_off;      // per state
    int n_gated;
    uint8_t tile_bit[kMaxTileBits];  // gated tile bits
    uint8_t qubit[kMaxTileBits];     // their global qubits
    uint16_t before[kMaxTileBits];   // tile bits un-rotated before this one in the backward sweep
};

// ---------------------------------------------------------------- particle-conserving ansatz
//
// Excitation gates exp(theta (T - T^dag)) (Sec. II-B, Eq. 5) with
// T = a_p^dag a_r or a_p^dag a_q^dag a_r a_s under the Jordan-Wigner mapping.
// T maps a basis state j with the annihilated modes occupied and the created
// ones empty to j' = j ^ (amask | cmask) with the sign
//     (-1)^(sign0 + popc(j & smask)),
// smask the xor of the "modes below" masks of the four (two) operators and
// sign0 the parity of the order relations between their modes.  A pass
// stages a tile of 2^k amplitudes (tile bits [0, m) = global bits [0, m),
// tile bits [m, k) = the pass's k - m further global bits, placed through a
// table of 2^(k-m) high-part offsets) and applies a run of consecutive gates
// whose modes all lie in the tile.

constexpr int kExcMaxGates = 16;      // gates of one pass
constexpr int kExcThreads = 256;

struct ExcGate {
    uint32_t amask, cmask;   // tile bits annihilated / created by T
    uint32_t smask_t;        // sign mask at tile bits (tile coordinates)
    uint32_t smask_g;        // sign mask at the global bits outside the tile
    uint32_t sign0;          // constant sign parity
    int n_fixed;             // 2 (single) or 4 (double)
    uint8_t fixed[4];        // tile bits of amask | cmask, increasing
    int param;               // parameter (and gate) index
};

struct ExcPass {
    int k, m;
    int g_begin, n_gates;    // gates [g_begin, g_begin + n_gates) of the gate table
    int hoff;                // first of the pass's 2^(k-m) high-part offsets
    uint32_t bmask;          // global bits taken from the tile number
    int grad_off;            // per-state column of the pass's gradient partials (tile-major)
    // Support of the state: the gates change only their own modes, so before
    // pass p every index that disagrees with psi_HF on a mode no earlier gate
    // touched holds zero.  A forward tile with (base & zmask) != zval is zero
    // (written as zeros by the first pass, skipped by later ones); a backward
    // tile with (base & bzmask) != bzval lies outside the support of the state
    // after this pass, so its gradient terms vanish and its lambda is never
    // read again (zero partials).
    uint32_t zmask, zval, bzmask, bzval;
};

template <typename T>
cudaError_t launch_exc_stage(const double *params, int n_exc, int batch, T *cs, cudaStream_t s);

template <typename T>
cudaError_t launch_exc_pass(const ExcPass &P, const ExcGate *gates_dev, const uint32_t *hoff_dev,
                            int n_qubits, int batch, void *psi, void *lam, size_t state_stride,
                            const T *cs, int n_exc, double *gpart, size_t grad_stride,
                            bool backward, int init_hf, uint64_t hf_index, cudaStream_t s);

// ---------------------------------------------------------------- Hamiltonian
//
// Terms grouped by x mask.  For a group with mask x and top bit h, every
// pair (i, i^x) with bit h of i clear contributes
//     2 * [ a * FA(i) + b * FB(i) ],   a + ib = conj(psi_i) psi_{i^x},
//     FA(i) = sum_{A terms} c' (-1)^{popc(i & z)},  FB likewise,
// where A terms have kappa = popc(x & z) even, B terms odd, and
// c' = c * (-1)^{floor(kappa/2)} (the phase (-i)^kappa of the Pauli string
// folded into a sign).  The x = 0 group contributes |psi_i|^2 FA(i).
struct GroupDesc {
    uint32_t x;
    int h;         // top bit of x (unused when x == 0)
    int t_begin;   // A terms: [t_begin, t_mid); B terms: [t_mid, t_end)
    int t_mid;
    int t_end;
};

// Per-state reduction layout of the energy kernels.
constexpr int kEnergyThreads = 256;
constexpr int kEnergyWinThreads = 512;

// One energy window: tile bits [0, m) and [m, k) -> global [a, a + k - m);
// groups wgroups[g_begin, g_end) are evaluated from the staged tile; block
// partials go to columns [block_off, block_off + 2^(n-k)).
// Window of the windowed expectation kernel.  Tile bits [0, m) are global
// bits [0, m); tile bits [m, k) are k - m further global bits in increasing
// order (any positions), placed through the window's table of 2^(k-m) high-part
// offsets; the tile number fills the remaining global bits `bmask` in
// increasing order.
struct WinDesc {
    int k, m;
    int g_begin, g_end;     // window groups [g_begin, g_end) (WinGroup array)
    int t_begin, t_count;   // window terms [t_begin, t_begin + t_count) (WinTerm array)
    int hoff;               // first of the window's 2^(k-m) high-part offsets
    uint32_t bmask;         // global bits taken from the tile number
    int block_off;          // first block-partial column of the window
    int with_norm;          // also yields <psi|psi> (the low window)
    int any_runs;           // some group uses the register-pattern transform
};

// Largest numbers of terms and groups of one window (staged in shared memory
// per tile) and of register patterns of a window group's terms.
constexpr int kWinMaxTerms = 2048;
constexpr int kWinMaxGroups = 96;
constexpr int kWinMaxRuns = 16;
constexpr int kWinDirectMax = 3;   // terms per class of a window group in direct mode

// A group inside a window.  Its terms are window-relative: A terms
// [a_begin, b_begin), B terms [b_begin, b_end), each class sorted by its
// register pattern v (the term's Z bits at the tile bits that distinguish a
// thread's pairs, or a thread's elements for the diagonal group xl == 0);
// arun[v] / brun[v] are the run starts relative to the class start and
// arun[NV] / brun[NV] the class length.
//
// In the expectation's windows a pair group may be split by the pattern of
// the bits of xl below its top bit (the top bit hl of i0 is always 0).  With
// those bits fixed, the terms merge per Z mask outside xl into one
// coefficient per pattern; the npat patterns whose coefficients do not all
// vanish are kept, pattern u fixing the tile bits `fmask` of i0 to fval[u].
// Pair P = tid + 512 s of a thread (slot s) has pattern u = P >> plog and free
// index f = P mod 2^plog, deposited around fmask: i0 = spread(f) | fval[u],
// spread(f) = sum_s (f & smask[s]) << s, and the bits of f at and above 9
// spread to dj[b] (0 beyond plog).  An unsplit group is the case npat = 1,
// fmask = 1 << hl.  Direct groups keep pattern u's class-A terms at
// a_begin + [arun[u], arun[u + 1]) and its class-B terms at
// b_begin + [brun[u], brun[u + 1]); run groups (unsplit) keep the runs above.
struct WinGroup {
    uint32_t xl;            // X mask in tile coordinates (0: the diagonal group)
    int hl;                 // top bit of xl
    int direct;             // 1: sign sums per pair, terms listed per pattern
    uint32_t fmask;         // fixed tile bits of i0 (expectation windows)
    int plog;               // log2 of the pairs per pattern
    int npat;               // patterns kept (direct groups)
    uint32_t fval[8];       // the fmask bits of i0 per pattern
    uint32_t smask[5];      // free-index bits moved up by s places in spread()
    uint32_t dj[4];         // spread of free-index bit 9 + b (0 beyond plog)
    int a_begin, b_begin, b_end;
    uint16_t arun[kWinMaxRuns + 1];
    uint16_t brun[kWinMaxRuns + 1];
};

// A term inside a window: its Z bits at tile positions (zt), its Z bits at
// tile-number positions (zout), and its sign-folded coefficient.
struct WinTerm {
    uint32_t zt, zout;
    double c;
};

// ---------------------------------------------------------------- sweeps
//
// lambda = H psi (and the expectation it yields) by sweeps over the whole
// state in a bit order chosen per sweep.  A sweep visits the basis states in
// the order of a counter s whose low bits run fastest: counter bit k is
// global bit order[k], with the low global bits [0, mlo) first (contiguous
// runs for coalescing), then the "fast" bits F of the sweep's groups, then
// the rest.  Every group of the sweep has its X mask inside [0, mlo) + F, so
// the partner psi_{i^x} of a state lies in the same block of 2^|F| states
// (the counter's low |F| + mlo bits), which all threads traverse together: a
// block is read from DRAM once and its gathers hit L2.  Per state i and
// group, lambda_i += psi_{i^x} (FA(i) - i FB(i)) with the sign sums FA, FB
// of the group's A and B terms at i.  The terms are merged per "pattern",
// the values of i at the group's X bits (up to kSweepMaxXBits of them):
// with z' = z & ~x,
//     FA(i) = sum_{z'} cA(pattern, z') (-1)^{popc(i & z')},
// so that most hopping-like groups need one term and no add per state, and
// patterns whose terms cancel (an XX + YY pair at equal bits) skip the
// gather.  Groups with more X bits keep their terms unmerged (one pattern).
constexpr int kSweepThreads = 256;
constexpr int kSweepJ = 4;             // states per thread and iteration
constexpr int kSweepChunk = 4096;      // counter values a block takes at a time
constexpr int kSweepFastBits = 20;     // low + fast bits: blocks of 2^20 states
constexpr int kSweepMaxXBits = 5;      // X bits of a group in pattern form
constexpr int kSweepMaxGroups = 256;   // per sweep
constexpr int kSweepMaxTerms = 4096;   // merged terms per sweep
constexpr int kSweepMaxPat = 8192;     // pattern offsets per sweep

struct SweepDesc {
    int g_begin, g_end;    // SGroup range
    int p_begin, n_pat;    // pattern offsets [p_begin, p_begin + n_pat)
    int t_begin, t_count;  // merged terms [t_begin, t_begin + t_count)
    int order;             // index of the sweep's 4 x 256 bit-order table
    int diag;              // 1: this sweep adds D_i psi_i (the diagonal of H)
    uint32_t fast;         // global bits of the counter's low part (informational)
};

// A group in a sweep.  Pattern p of a state i is bit ((xbits >> 5k) & 31)
// of i at bit k of p (k < nxb).  When no pattern has more than one merged
// term, pattern p's term is term slot pat + p of the sweep (a zero term for
// an empty pattern).  Otherwise ("multi") entry p of the group's pattern
// array (at offset `pat` of the sweep's) is first | count << 16: its merged
// terms [first, first + count), sweep-relative.  "Parity" groups (the
// nonempty patterns are those of one parity p of the X bits and share one
// merged term) keep that term in slot pat alone: a state takes it when
// popc(i & x) has parity p.  flags: nxb | has_b << 8 (class-B terms) |
// multi << 9 | parity form << 10 | p << 11.
struct SGroup {
    uint32_t x;
    int pat;
    uint32_t xbits;
    uint32_t flags;
};

// ---------------------------------------------------------------- launchers
// Each returns cudaGetLastError() after queueing.

template <typename T>
cudaError_t launch_stage(const StageSlot *slots_dev, int n_slots, int n_qubits, int depth,
                         const double *params, int batch, RotCoef<T> *coefs, size_t coef_stride,
                         void *dtab, size_t dtab_stride, cudaStream_t s);

template <typename T>
cudaError_t launch_pass(const PassDesc *desc_dev, const PassDesc &desc_host, int n_qubits,
                        int batch, void *psi, void *lam, size_t state_stride,
                        const RotCoef<T> *coefs, size_t coef_stride, const void *dtab,
                        size_t dtab_stride, double *grad_part, size_t grad_stride, bool backward,
                        int init_zero, cudaStream_t s);

template <typename T>
cudaError_t launch_energy(const GroupDesc *groups, int n_groups, const uint32_t *tz,
                          const double *tc, const void *hdiag, int n_qubits, int batch,
                          const void *psi, size_t state_stride, double *partials,
                          int blocks_per_state, cudaStream_t s);

template <typename T>
cudaError_t launch_apply_h(const GroupDesc *groups, int n_groups, const uint32_t *tz,
                           const double *tc, const void *hdiag, int n_qubits, int batch,
                           const void *psi, void *lam, size_t state_stride, double *partials,
                           int blocks_per_state, cudaStream_t s);

template <typename T>
cudaError_t launch_energy_win(const WinDesc &W, const WinGroup *wgroups, const WinTerm *wterms,
                              const uint32_t *hoff, const void *hdiag, int n_qubits, int batch,
                              const void *psi, size_t state_stride, double *partials,
                              int bps_total, cudaStream_t s);
// Windowed apply-H over windows planned with each group's terms ordered by
// their pattern over a thread's elements: `first` writes lambda, later windows
// add to it; the `last` window writes block partials (Re<psi|lambda>, norm)
// at [state][blockIdx.x] with 2^(n - W.k) columns per state.
template <typename T>
cudaError_t launch_apply_h_win(const WinDesc &W, const WinGroup *wgroups, const WinTerm *wterms,
                               const uint32_t *hoff, const void *hdiag, int n_qubits, int batch,
                               const void *psi, void *lam, size_t state_stride, int first,
                               int last, double *partials, cudaStream_t s);
// Sweep form of apply-H: `first` writes lambda, later sweeps add to it; the
// `last` sweep writes chunk partials (Re<psi|lambda>, norm, 0) at
// cpart[(state * nchunks + chunk) * 3], nchunks = ceil(2^n / kSweepChunk).
// `ctr` holds one zeroed counter per state for this launch.  `order` points
// at the sweep's 1024-entry bit-order table; terms, groups and patterns are
// the whole plan's arrays (the sweep's ranges are in W); coefficients are T.
// `blocks` blocks per state.
template <typename T>
cudaError_t launch_apply_h_sweep(const SweepDesc &W, const uint32_t *order, const SGroup *groups,
                                 const uint32_t *pat, const uint32_t *tz, const void *ca,
                                 const void *cb, const void *hdiag, int n_qubits, int batch,
                                 const void *psi, void *lam, size_t state_stride, int first,
                                 int last, unsigned long long *ctr, double *cpart, int blocks,
                                 cudaStream_t s);
size_t sweep_smem_bytes(const SweepDesc &W, size_t real_bytes);
int sweep_blocks_per_sm(int elem_bytes, size_t smem);
// Tile bits (log2 of elements) of the windowed expectation for a precision:
// 512 threads hold 2^(kWinBits - 9) elements each.
constexpr int win_tile_bits(bool c128) { return c128 ? 12 : 13; }

// Diagonal of H from the x = 0 group's terms (z masks, FP64 coefficients with
// the Pauli phase folded): D[i] for i < 2^n_qubits, stored as T.  `hdiag`
// arguments of the expectation kernels may be null (terms evaluated inline).
template <typename T>
cudaError_t launch_build_hdiag(const uint32_t *z, const double *c, int n_terms, int n_qubits,
                               void *D, int sms, cudaStream_t s);
template <typename T>
cudaError_t launch_energy_sub(const GroupDesc *groups, int n_groups, const uint32_t *tz,
                              const double *tc, int n_qubits, int batch, const void *psi,
                              size_t state_stride, double *partials, int bps, int block_off,
                              int bps_total, cudaStream_t s);

cudaError_t launch_energy_finish(const double *partials, int blocks_per_state, int batch,
                                 double *energies, double *norms, double *unnorm,
                                 cudaStream_t s);

// Gradient reduction: param p of state b sums `count` partials at
// part[b*stride + off[p] + j*step], j = 0..count-1.
cudaError_t launch_grad_finish(const double *part, size_t part_stride, const int *off,
                               const int *count, const int *step, int n_params, int batch,
                               double *grads, cudaStream_t s);

// One gate per pass (reference kernel): RY/RZ on qubit q, or CZ(q, q+1).
template <typename T>
cudaError_t launch_gate_ry(void *psi, size_t stride, int n, int batch, int q, const double *params,
                           int pidx, int pstride, cudaStream_t s);
template <typename T>
cudaError_t launch_gate_rz(void *psi, size_t stride, int n, int batch, int q, const double *params,
                           int pidx, int pstride, cudaStream_t s);
template <typename T>
cudaError_t launch_gate_cz(void *psi, size_t stride, int n, int batch, int q, cudaStream_t s);
template <typename T>
cudaError_t launch_init_zero_state(void *psi, size_t stride, int n, int batch, cudaStream_t s);

int pass_threads(const PassDesc &d);
size_t pass_smem_bytes(const PassDesc &d, bool backward, size_t elem_bytes);

}  // namespace vqe
