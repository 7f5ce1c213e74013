/*
 * kin_peaks.h -- C ABI of the arithmetic-peak probe (libkin_peaks.so).
 *
 * The integrator's hot path is bound by the GPU's FP64 pipe (and, for the
 * mixed-precision path, possibly its FP32 pipe), not by memory bandwidth:
 * every cell moves a few hundred bytes per call but needs 1e5..1e8
 * floating-point operations (Sections 3.1-3.4 of Niemeyer & Sung measure
 * this path as arithmetic-heavy per-thread integration). The roofline of the
 * benchmark therefore divides by the pipe's measured fused multiply-add
 * rate, which this probe measures on the current device.
 *
 * The paper has no counterpart of this probe (it reports speedups only).
 */
#ifndef KIN_PEAKS_H
#define KIN_PEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KINPK_FP64 0
#define KINPK_FP32 1

/* Run `blocks_per_sm` x (SM count) blocks of `threads` threads (a multiple
 * of 32, <= 1024), each thread advancing 8 independent chains of `iters`
 * dependent fused multiply-adds x <- x a + b in the given precision, on
 * `stream` (a cudaStream_t; NULL = legacy default). Synchronous: returns
 * after the kernel ends. Outputs: *ms, the kernel's duration from CUDA events
 * on that stream; *fma_per_s, fused multiply-adds per second over the whole
 * device (flops per second are twice this). Both pointers are host memory.
 * Returns 0, -1 for a bad argument (precision, threads, iters < 1,
 * blocks_per_sm < 1, NULL outputs), -3 when a CUDA call fails
 * (kinpk_last_error() gives the CUDA error string). No device memory is
 * allocated beyond the launch itself. */
int kinpk_fma_rate(int32_t precision, int64_t iters, int32_t blocks_per_sm, int32_t threads,
                   void *stream, double *ms, double *fma_per_s);

/* Message of the last failed call on this thread ("" if none). */
const char *kinpk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KIN_PEAKS_H */
