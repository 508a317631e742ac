/*
 * ostrich_probe.h -- measurement helper of libostrich.  The paper has no counterpart:
 * this is not part of the method.  It measures the FP32 fused multiply-add throughput
 * of the GPU, the denominator of the step kernel's ALU roofline (the step kernel is
 * bound by plain FP32 arithmetic, not by HBM or the tensor cores).
 */
#ifndef OSTRICH_PROBE_H
#define OSTRICH_PROBE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Runs an FFMA-only kernel (eight independent dependency chains per thread, grid of
 * blocks_per_sm x SMs blocks of 1024 threads, `iters` x 128 FFMAs per thread) once
 * untimed and `reps` times timed with CUDA events on `stream`.  out: caller-owned
 * device buffer of at least n_threads floats (blocks_per_sm x SMs x 1024), written with
 * each thread's final value so the chains stay live.  On success *tflops receives the
 * achieved FP32 TFLOP/s (2 flops per FFMA), *ms the mean kernel time and *n_threads
 * the thread count used.  Returns 0, or a CUDA error code (non-zero) on failure; with
 * out == NULL it only reports the thread count the call would use. */
int ostrich_probe_ffma(int blocks_per_sm, int iters, int reps, float* out, size_t* n_threads, double* tflops,
                       double* ms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OSTRICH_PROBE_H */
