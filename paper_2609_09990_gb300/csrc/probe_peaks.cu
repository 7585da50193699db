// Arithmetic peak probe: independent FMA chains on every SM, timed with CUDA
// events.  Gives the FP64 and FP32 CUDA-core rates that bound the FP64 path
// (GB300 has no fast FP64 tensor path).
#include <cuda_runtime.h>

#include "../../include/gbdmrg_test.h"

namespace {
template <class T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <class T>
double rate(int iters, int sms) {
  int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0);
  for (int r = 0; r < 5; ++r) fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return 5.0 * blocks * threads * (double)iters * 16.0 / (ms / 1e3) / 1e12;
}
}  // namespace

extern "C" int gbd_probe_peaks(int32_t device, double* fp64_tflops, double* fp32_tflops) {
  if (cudaSetDevice(device) != cudaSuccess) return GBD_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (fp64_tflops) *fp64_tflops = rate<double>(20000, sms);
  if (fp32_tflops) *fp32_tflops = rate<float>(200000, sms);
  return cudaGetLastError() == cudaSuccess ? GBD_OK : GBD_ERR_CUDA;
}
