/*
 * st_probe.h -- device arithmetic peak probes (no counterpart in the paper).
 *
 * The roofline fractions of kernels bound by the FP64 or FP32 pipes (the
 * combination sum, the time transforms, the FP64 stencils) are taken against
 * the rate these probes measure on the current device, not a nominal figure.
 */
#ifndef ST_PROBE_H_
#define ST_PROBE_H_

#include "st.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Sustained fused multiply-add rate of the current device in GFLOP/s (one FMA
 * counted as two flops): eight 256-thread CTAs per SM, each thread running
 * eight independent FMA chains of iters x 16 steps (iters x 128 FMAs per
 * thread), timed with CUDA events on `stream` after one short warm-up launch.
 * precision: 0 = FP64, 1 = FP32.  *gflops is written on the host; the call
 * synchronises the stream.  Allocates one small output buffer with
 * cudaMallocAsync on `stream` (ST_ERR_OOM if that fails); ST_ERR_ARG for
 * iters outside 1..2^24 or another precision; ST_ERR_CUDA if a launch fails. */
st_status st_probe_fma(int precision, int iters, double* gflops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ST_PROBE_H_ */
