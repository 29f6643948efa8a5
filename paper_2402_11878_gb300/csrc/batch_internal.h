// Internal records of the batched driver (k_batch.cu, vqe_batch.cu).
#pragma once

#include "vqe_internal.h"

namespace vqe {

constexpr int kBatchThreads = 512;
constexpr int kBatchMaxSlots = 48;     // staging slots of one instance's plan
constexpr int kBatchMaxPasses = 64;

struct BatchPlan {
    int n, depth;
    int pass_off, n_passes;      // into the forward/backward pass arrays
    int stage_off, n_stage;      // into the staging-slot array
    int slot_first[kBatchMaxPasses];  // first staging slot of each pass
    int coef_entries;            // coefficient rows of all slots (entries)
    int kl, lo_stride, hi_stride;     // diagonal half tables
    int whole_tile;              // every pass spans all qubits: the state stays in shared memory
};

struct BatchInst {
    int index;          // position in the caller's arrays
    int n, depth, plan;
    size_t params_off;  // offset of this instance's parameters (and gradient)
    int groups_off, n_groups, terms_off;
};

struct BatchLayout {   // dynamic shared memory offsets (bytes)
    size_t off_psi, off_lam, off_gsh, off_coef, off_lo, off_hi, off_gacc, off_red, off_slotbase;
    size_t off_phc, off_phs, off_scl, off_sigma;
    size_t total;
};

struct BatchArgs {
    const BatchInst *inst;
    const int *order;
    int count;
    int *counter;
    const BatchPlan *plans;
    const PassDesc *fwd, *bwd;
    const StageSlot *stage;
    const GroupDesc *groups;
    const uint32_t *tz;
    const void *tc;
    const double *params;
    double *energies, *grads;
    void *scratch;          // per CTA: psi and lambda slices of scratch_elems amplitudes
    size_t scratch_elems;
    BatchLayout layout;
};

// r4: the kernel for instances whose plans hold 16 amplitudes per thread
// (R = 4); the other kernel takes R <= 3.
template <typename T>
cudaError_t launch_batch(const BatchArgs &args, bool r4, int grid, size_t smem, cudaStream_t s);

}  // namespace vqe
