// FP32 FFMA throughput probe (declared in include/ostrich_probe.h): the measured
// denominator of the step kernel's ALU roofline.  Not part of the method.
#include <cuda_runtime.h>

#include "ostrich_probe.h"

namespace {

// Eight independent FFMA chains per thread, 16 rounds unrolled per iteration: 128
// FFMAs per iteration.  x -> x * b + c with b just below 1 keeps every value normal and
// bounded, so no chain can be folded away or hit slow paths.
__global__ void __launch_bounds__(1024) ffma_probe_kernel(float* out, int iters, float seed) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float a0 = seed + 1e-6f * (float)(threadIdx.x & 63), a1 = a0 + 0.1f, a2 = a0 + 0.2f, a3 = a0 + 0.3f;
  float a4 = a0 + 0.4f, a5 = a0 + 0.5f, a6 = a0 + 0.6f, a7 = a0 + 0.7f;
  const float b = 0.99999994f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = fmaf(a0, b, c); a1 = fmaf(a1, b, c); a2 = fmaf(a2, b, c); a3 = fmaf(a3, b, c);
      a4 = fmaf(a4, b, c); a5 = fmaf(a5, b, c); a6 = fmaf(a6, b, c); a7 = fmaf(a7, b, c);
    }
  }
  out[t] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

}  // namespace

extern "C" int ostrich_probe_ffma(int blocks_per_sm, int iters, int reps, float* out, size_t* n_threads,
                                  double* tflops, double* ms, void* stream) {
  if (blocks_per_sm < 1 || iters < 1 || reps < 1 || !n_threads) return (int)cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int blocks = blocks_per_sm * sms, threads = 1024;
  *n_threads = (size_t)blocks * threads;
  if (!out) return 0;
  if (!tflops || !ms) return (int)cudaErrorInvalidValue;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ffma_probe_kernel<<<blocks, threads, 0, st>>>(out, iters, 1.0f);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return (int)e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return (int)e; }
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps; ++r) ffma_probe_kernel<<<blocks, threads, 0, st>>>(out, iters, 1.0f + 1e-3f * r);
  cudaEventRecord(e1, st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return (int)e;
  *ms = (double)t / reps;
  const double flops = 2.0 * 128.0 * (double)iters * (double)(*n_threads);
  *tflops = flops / (*ms * 1e-3) / 1e12;
  return 0;
}
