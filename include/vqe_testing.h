/*
 * vqe_testing.h -- fault injection for the tests of libvqe_gb300.
 *
 * The error contract of include/vqe.h says that a failed call leaves the
 * handle's Hamiltonian, state and workspace as they were.  Device memory
 * rarely runs out in a test, so this hook makes the library's own device
 * allocations fail on the host, without touching the GPU: the failing
 * allocation returns VQE_ERR_OOM exactly as a failed cudaMalloc does.  It is
 * test support with no counterpart in the paper.
 */
#ifndef VQE_GB300_TESTING_H
#define VQE_GB300_TESTING_H

#ifdef __cplusplus
extern "C" {
#endif

/* after >= 0: the next `after` device allocations the library makes succeed
 * and every one after them fails with VQE_ERR_OOM (process-wide, all
 * handles); after < 0: no injected failures (the default).  Allocations of
 * the batched driver and of the measurement probe are not affected. */
void vqe_testing_fail_allocations(int after);

#ifdef __cplusplus
}
#endif
#endif
