// th_coarse_solve_noalloc: the FP64 coarse block solve with its scratch in a
// fixed device array of this library instead of the context's workspace.
//
// The coarse block sweep keeps the forward-sweep block vectors z_j (one
// complex value per coarse node and right-hand side) between its forward
// and backward passes.  This entry point keeps them in g_noalloc_z below, a
// file-scope device array that every GPU loading the library holds until the
// process exits, so a call needs no memory beyond the caller's input and
// output vectors and the context's read-only factors.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"
#include "th_internal.h"

namespace th {
bool coarse_factors_fp64(const th_ctx* ctx, CoarseSolveArgs<double>* a, int* cluster, int* nrhs_max, int* device);
}

namespace {

// Capacity: 2^18 complex FP64 values (4 MiB), i.e. Nc * nrhs <= 262144
// (a 401 x 401 coarse grid holds 160801 values, a 201 x 201 grid 40401).
constexpr long long kNoallocComplex = 1LL << 18;

static __device__ __align__(256) double2 g_noalloc_z[kNoallocComplex];

// Device address of g_noalloc_z.  Host code must not use the symbol itself as
// a device pointer.  The address is looked up with the caller's device current
// on every call made outside a stream capture, so a module reload (after a
// device reset, or with another context current) cannot leave a stale pointer
// behind; the copy kept per device is used only while the caller's stream is
// being captured, when a lookup could load the module and is not allowed.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2* g_addr[kMaxDevices] = {};

th_status scratch_address(int dev, cudaStream_t stream, double2** out) {
  if (dev < 0 || dev >= kMaxDevices) return TH_ERR_CUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return TH_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cap != cudaStreamCaptureStatusNone) {
    if (!g_addr[dev]) return TH_ERR_CUDA;  // first call on this device inside a capture
    *out = g_addr[dev];
    return TH_OK;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_z) != cudaSuccess || !p) return TH_ERR_CUDA;
  g_addr[dev] = static_cast<double2*>(p);
  *out = g_addr[dev];
  return TH_OK;
}

}  // namespace

extern "C" th_status th_coarse_solve_noalloc(const th_ctx* ctx, const double* rc_dev, double* uc_dev, int nrhs,
                                             void* stream) {
  if (!ctx || !rc_dev || !uc_dev || nrhs < 1) return TH_ERR_ARG;
  th::CoarseSolveArgs<double> a{};
  int cluster = 0, nrhs_max = 0, ctx_dev = -1;
  if (!th::coarse_factors_fp64(ctx, &a, &cluster, &nrhs_max, &ctx_dev)) return TH_ERR_UNSUPPORTED;
  if (nrhs > nrhs_max) return TH_ERR_ARG;
  if (a.Nc * (long long)nrhs > kNoallocComplex) return TH_ERR_ARG;  // beyond the fixed scratch
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TH_ERR_CUDA;
  if (dev != ctx_dev) return TH_ERR_ARG;  // the factors live on another device
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double2* z = nullptr;
  th_status st = scratch_address(dev, s, &z);
  if (st != TH_OK) return st;
  a.rhs = reinterpret_cast<const double2*>(rc_dev);
  a.x = reinterpret_cast<double2*>(uc_dev);
  a.z = z;  // every z entry is written by the forward sweep before the backward sweep reads it
  cudaError_t e = th::launch_coarse_solve<double>(a, nrhs, cluster, s);
  return e == cudaSuccess ? TH_OK : TH_ERR_CUDA;
}
