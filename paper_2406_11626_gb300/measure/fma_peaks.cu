// Throughput probe for the plain (non-tensor) FP64 and FP32 FMA pipes.
//
// The CCZ4 right-hand side is a stencil followed by pointwise tensor algebra:
// it is not a dense contraction, so its roofline is set by the scalar FMA
// pipes, not by the tensor cores. This probe measures that ceiling on the
// device it runs on: every thread runs eight independent FMA chains, so the
// pipe (not the dependency latency) is the limit.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

template <typename T>
__global__ void fma_chains(T *out, int iters, T m, T c) {
  T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
      a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
    }
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

template <typename T>
int run(int blocks_per_sm, int iters, double *tflops, double *ms_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 3;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 3;
  const int threads = 256;
  const int blocks = sms * blocks_per_sm;
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // one untimed launch to load the module and settle clocks
  fma_chains<T><<<blocks, threads>>>(out, iters / 8 + 1, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0);
  fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  int rc = cudaGetLastError() == cudaSuccess ? 0 : 3;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  const double flops = 2.0 * 8.0 * 4.0 * (double)iters * (double)blocks * threads;
  if (tflops) *tflops = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return rc;
}

}  // namespace

// Measures the FMA throughput of the FP64 (precision = 64) or FP32
// (precision = 32) pipe on the current device, in TFLOP/s (an FMA counts as
// two flops). Returns 0 on success, 1 on a bad argument, 2 if the small output
// buffer cannot be allocated, 3 on a CUDA error.
extern "C" int ccz4_probe_fma_rate(int precision, int blocks_per_sm, int iters,
                                   double *tflops, double *ms) {
  if (blocks_per_sm <= 0 || iters <= 0) return 1;
  if (precision == 64) return run<double>(blocks_per_sm, iters, tflops, ms);
  if (precision == 32) return run<float>(blocks_per_sm, iters, tflops, ms);
  return 1;
}
