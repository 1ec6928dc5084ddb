/* regc_probe.h -- measurement tooling, not part of the method.
 *
 * The sweep kernel's roofline fraction is quoted against the FP32 pipe's
 * peak, which the device-wide measured peaks do not list.  This entry point
 * measures it on the GPU at hand.  It lives in its own shared library,
 * libregc_probe.so (built beside libregc.so), which only the benchmark loads.
 */
#ifndef REGC_PROBE_H
#define REGC_PROBE_H

#include "regc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* FP32 peak of the current GPU, measured: an FFMA-loop kernel (8 independent
 * chains per thread, 8 CTAs of 256 threads per SM, `iters` x 128 FMA per
 * thread) timed with CUDA events on cuda_stream after one warm-up launch.
 * *tflops receives 2 x FMAs / time in TFLOP/s.  Synchronous.  Errors:
 * REGC_EINVAL (iters < 1, tflops NULL), REGC_ECUDA (a CUDA call failed). */
REGC_API regc_status regc_probe_fp32_peak(int iters, void *cuda_stream, double *tflops);

#ifdef __cplusplus
}
#endif

#endif
