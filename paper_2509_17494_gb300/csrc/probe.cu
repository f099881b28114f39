// Arithmetic peak probes (measurement only, not on the two-grid path).
//
// The FP64 form's subdomain products and coarse sweeps are bound by the FP64
// pipe, the mixed form's double-single residual by the FP32 pipe; their
// roofline fractions need the rate those pipes reach on this GPU.  Each probe
// launches a few blocks per SM whose threads run 8 independent chains of
// dependent fused multiply-adds x <- x a + b (2 flops each) and times them
// with CUDA events; the result of every chain is kept live.
#include <cuda_runtime.h>

#include "th.h"

namespace {

__device__ double g_sink[8];  // target of the never-taken store that keeps the chains live

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == (T)-1) out[blockIdx.x & 7] = s;  // never true for these inputs; keeps the chains live
}

template <typename T>
th_status probe(int iters, double* flops_per_s, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TH_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TH_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  void* sink = nullptr;
  if (cudaGetSymbolAddress(&sink, g_sink) != cudaSuccess) return TH_ERR_CUDA;
  T* out = static_cast<T*>(sink);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TH_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return TH_ERR_CUDA;
  }
  const T a = (T)0.999999, b = (T)1e-6;
  k_fma_chains<T><<<blocks, threads, 0, s>>>(out, iters / 10 + 1, a, b);  // warm-up
  cudaEventRecord(e0, s);
  k_fma_chains<T><<<blocks, threads, 0, s>>>(out, iters, a, b);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) return TH_ERR_CUDA;
  *flops_per_s = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
  return TH_OK;
}

}  // namespace

extern "C" th_status th_peak_fma(int prec, int iters, double* flops_per_s, void* stream) {
  if (!flops_per_s || iters < 1) return TH_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (prec == TH_PREC_FP64) return probe<double>(iters, flops_per_s, s);
  if (prec == TH_PREC_FP32) return probe<float>(iters, flops_per_s, s);
  return TH_ERR_ARG;
}
