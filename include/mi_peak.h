/*
 * mi_peak.h -- ALU throughput microbenchmark of libmi_delbm (the paper has no
 * counterpart: it measures the denominators of the library's ALU rooflines on
 * the GPU it runs on, instead of taking nominal unit counts and clocks).
 */
#ifndef MI_PEAK_H
#define MI_PEAK_H

#include "mi_delbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Dense fused multiply-add throughput of the current device.
 *
 * precision: 0 = FP32, 1 = FP64.  The kernel runs one CTA of 256 threads per
 * resident slot on every SM (as many as fit), each thread 8 independent
 * dependency chains of x <- fma(x, a, b), long enough to take about 20 ms;
 * a first launch warms up the clocks and is not timed.  Each FMA counts as
 * 2 FLOP.  Timed with CUDA events on `stream` (cudaStream_t, NULL = default
 * stream); the call synchronises that stream.
 * tflops_out: measured TFLOP/s; ms_out (may be NULL): the timed launch's
 * duration.  Allocates 4 bytes x threads of device memory for the results
 * (they are kept only so that the chains are not optimised away) and frees it.
 * Errors (message via mi_delbm_last_error(NULL)): MI_EINVAL (precision not 0
 * or 1, tflops_out NULL), MI_ENOMEM, MI_ECUDA. */
mi_status mi_measure_fma_peak(int precision, double *tflops_out, double *ms_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MI_PEAK_H */
