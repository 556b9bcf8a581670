// Arithmetic-peak microbenchmark: independent register-resident fused
// multiply-add chains over the whole GPU.  Its FP64 figure is the roofline
// denominator of the FP64 integrator, which is bound by the FP64 pipe.
#include <cuda_runtime.h>

#include "qcams.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, int iters, T a, T b) {
  T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == (T)-12345) out[blockIdx.x] = s;   // keeps the chains live
}

template <typename T>
int run_peak(int iters, double* flops, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QCAMS_E_NODEVICE;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return QCAMS_E_NODEVICE;
  const int block = 256, grid = sms * 8;
  T* out = nullptr;
  if (cudaMallocAsync(&out, sizeof(T) * grid, st) != cudaSuccess) return QCAMS_E_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_chains<T><<<grid, block, 0, st>>>(out, iters / 8 + 1, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0, st);
  k_fma_chains<T><<<grid, block, 0, st>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (e != cudaSuccess || ms <= 0.f) return QCAMS_E_CUDA;
  const double fl = 2.0 * 32.0 * (double)iters * (double)block * (double)grid;
  *flops = fl / (ms * 1e-3);
  return QCAMS_OK;
}

}  // namespace

extern "C" int qcams_fma_peak(int32_t precision, double* flops_per_s, void* cuda_stream) {
  if (!flops_per_s || (precision != 64 && precision != 32)) return QCAMS_E_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (precision == 64) return run_peak<double>(4096, flops_per_s, st);
  return run_peak<float>(131072, flops_per_s, st);
}
