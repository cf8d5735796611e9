// Measured ALU roofline of this GPU: fused multiply-add throughput in FP64
// and FP32 (a measurement aid for the ALU-bound FP64 kernels).
#include "internal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; k++) x[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) s += x[k];
  if (s == (T)-12345.0) out[threadIdx.x] = s;  // keeps the chain alive
}

template <typename T>
int run(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, iters = 8192;
  T* out = nullptr;  // sink for the (never taken) store that keeps the chains live
  if (cudaMallocAsync((void**)&out, 256 * sizeof(T), st) != cudaSuccess) {
    cudaGetLastError();
    return LQCD_ENOMEM;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LQCD_ECUDA;
  k_fma_peak<T><<<blocks, 256, 0, st>>>(out, iters / 8, (T)0.999999, (T)1e-7);  // warm-up
  cudaEventRecord(e0, st);
  k_fma_peak<T><<<blocks, 256, 0, st>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1, st);
  lq_count_launch();
  lq_count_launch();
  if (cudaEventSynchronize(e1) != cudaSuccess) return LQCD_ECUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  const double flops = 2.0 * 8.0 * iters * (double)blocks * 256.0;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return cudaGetLastError() == cudaSuccess ? 0 : LQCD_ECUDA;
}

}  // namespace

extern "C" int lqcd_fma_peak(int bits, double* tflops, void* stream) {
  if (!tflops || (bits != 64 && bits != 32)) {
    lq_set_error("fma_peak: bits must be 64 or 32");
    return LQCD_EBADARG;
  }
  return bits == 64 ? run<double>(tflops, (cudaStream_t)stream) : run<float>(tflops, (cudaStream_t)stream);
}
