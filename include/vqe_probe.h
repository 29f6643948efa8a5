/*
 * vqe_probe.h -- measured arithmetic peak of the current GPU.
 *
 * The FP64 tile passes of the ansatz are bound by the FP64 fused
 * multiply-add rate rather than by memory bandwidth, so their roofline needs
 * a measured FMA peak.  This call measures it.  It is measurement support
 * with no counterpart in the paper.
 */
#ifndef VQE_GB300_PROBE_H
#define VQE_GB300_PROBE_H

#include "vqe.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Measure the FMA throughput of the current device: fp64 = 1 for FP64,
 * 0 for FP32.  Launches one untimed and one timed kernel of independent FMA
 * chains on every SM (8 blocks of 256 threads per SM) on cuda_stream (NULL =
 * legacy default stream), timed with CUDA events, and writes the rate in
 * TFLOP/s (2 flops per FMA) to *tflops.  Allocates and frees a small output
 * buffer (8 bytes per thread); synchronises the stream.  Changes no clock or
 * power setting.  Errors: VQE_ERR_ARG (NULL output, fp64 not 0/1),
 * VQE_ERR_OOM, VQE_ERR_CUDA. */
vqe_status vqe_measure_fma_peak(int fp64, void *cuda_stream, double *tflops);

#ifdef __cplusplus
}
#endif
#endif
