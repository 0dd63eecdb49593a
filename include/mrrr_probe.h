/*
 * mrrr_probe.h -- device-throughput probe used to put the solver's kernels on
 * a roofline.  The paper has no counterpart: it measures the machine, not the
 * method.
 *
 * The solver's recurrences are bound by the binary64 (FP64) pipe of the SMs,
 * whose rate is not part of the device attributes.  This call measures it:
 * one launch of 8 warps per SM (one CTA of 256 threads per SM) in which
 * every thread runs 8 independent chains of `iters` dependent binary64 fused
 * multiply-adds, timed with CUDA events on `stream`.
 *
 *   *gflops  receives 2 * (threads * 8 * iters) / seconds / 1e9
 *   *ms      receives the launch's device time in milliseconds
 *
 * iters <= 0 selects 65536.  The launch runs twice (the first warms the
 * clocks up) and the second is reported.  Returns 0, MRRR_ERR_ARG for NULL
 * outputs or MRRR_ERR_CUDA.  Work and events are enqueued on `stream` and the
 * call synchronises it before returning.
 */
#ifndef MRRR_PROBE_H
#define MRRR_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

int mrrr_probe_fp64_fma(int iters, double* gflops, double* ms, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MRRR_PROBE_H */
