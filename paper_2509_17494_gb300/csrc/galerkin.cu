// Galerkin p-type coarsening (Section 4, the paper's comparison method 'gal'):
// the coarse operator A_c = I_P^T A_{alpha_c} I_P is the Q_{p/2} finite-element
// operator on the fine mesh, stored as a (2q+1)^2-point stencil per coarse
// node (q = p/2), and solved by a block forward / backward sweep over groups of
// q coarse node rows with the FP64 set-up's explicit block inverses G_j.
//   K15 k_gal_apply: y = A_c x, one thread per (node, rhs).
//   K16 k_gal_step:  one block step of the sweep.  Every CTA forms the coupled
//                    right-hand side t of block j in shared memory (the stencil
//                    terms that reach the neighbouring group), then its warps
//                    take rows of G_j: forward x_j = G_j (b_j - L_j x_{j-1}),
//                    backward x_j -= G_j U_j x_{j+1}.
#include "kernels.h"

namespace th {

template <typename C>
__device__ __forceinline__ void gal_fma(C& acc, C a, C b) {
  cmadd(acc, a, b);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gal_apply(const GalArgs<T> a) {
  using C = typename Cx<T>::t;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= a.Nc) return;
  const int rhs = blockIdx.y;
  const int q = a.q, mc = a.mc, S = 2 * q + 1;
  const int y = (int)(node / mc), x = (int)(node % mc);
  const C* X = a.b + (size_t)rhs * a.Nc;
  const C* st = a.st + (size_t)node * S * S;
  C acc;
  acc.x = 0;
  acc.y = 0;
  const int dy0 = max(-q, -y), dy1 = min(q, mc - 1 - y), dx0 = max(-q, -x), dx1 = min(q, mc - 1 - x);
  for (int dy = dy0; dy <= dy1; ++dy)
    for (int dx = dx0; dx <= dx1; ++dx)
      gal_fma(acc, st[(dy + q) * S + dx + q], X[(size_t)(y + dy) * mc + x + dx]);
  a.x[(size_t)rhs * a.Nc + node] = acc;
}

template <typename T>
__global__ void __launch_bounds__(256) k_gal_step(const GalArgs<T> a, int j, int backward) {
  using C = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char gal_sm[];
  C* t = reinterpret_cast<C*>(gal_sm);
  const int q = a.q, mc = a.mc, S = 2 * q + 1;
  const int lo = gal_row_lo(j, q), hi = gal_row_hi(j, q);
  const int Sj = (hi - lo + 1) * mc;
  const size_t off = (size_t)lo * mc;
  const int rhs = blockIdx.y;
  const C* X = a.x + (size_t)rhs * a.Nc;
  // the rows of the group the coupling reads
  int nlo = 0, nhi = -1;
  if (!backward && j > 0) {
    nlo = gal_row_lo(j - 1, q);
    nhi = lo - 1;
  } else if (backward && j + 1 < a.nblk) {
    nlo = hi + 1;
    nhi = gal_row_hi(j + 1, q);
  }
  for (int i = threadIdx.x; i < Sj; i += blockDim.x) {
    const int y = lo + i / mc, x = i % mc;
    const C* st = a.st + (off + i) * S * S;
    C acc;
    acc.x = 0;
    acc.y = 0;
    const int dy0 = max(-q, nlo - y), dy1 = min(q, nhi - y), dx0 = max(-q, -x), dx1 = min(q, mc - 1 - x);
    for (int dy = dy0; dy <= dy1; ++dy)
      for (int dx = dx0; dx <= dx1; ++dx)
        gal_fma(acc, st[(dy + q) * S + dx + q], X[(size_t)(y + dy) * mc + x + dx]);
    if (backward) {
      t[i] = acc;
    } else {
      const C bv = a.b[(size_t)rhs * a.Nc + off + i];
      C v;
      v.x = bv.x - acc.x;
      v.y = bv.y - acc.y;
      t[i] = v;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  const C* G = a.G + gal_goff(j, q, mc);
  C* Xo = a.x + (size_t)rhs * a.Nc + off;
  for (int row = blockIdx.x * warps + (threadIdx.x >> 5); row < Sj; row += gridDim.x * warps) {
    const C* g = G + (size_t)row * Sj;
    C acc;
    acc.x = 0;
    acc.y = 0;
#pragma unroll 4
    for (int c = lane; c < Sj; c += 32) gal_fma(acc, g[c], t[c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
      if (backward) {
        C z = Xo[row];
        z.x -= acc.x;
        z.y -= acc.y;
        Xo[row] = z;
      } else {
        Xo[row] = acc;
      }
    }
  }
}

template <typename T>
cudaError_t launch_gal_apply(const GalArgs<T>& a, cudaStream_t s) {
  const dim3 grid((unsigned)((a.Nc + 255) / 256), a.nrhs);
  k_gal_apply<T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

int gal_solve_launches(int nblk) { return 2 * nblk - 1; }

template <typename T>
cudaError_t launch_gal_solve(const GalArgs<T>& a, cudaStream_t s) {
  using C = typename Cx<T>::t;
  const int smax = (a.q + 1) * a.mc;  // the largest block (block 0)
  const size_t smem = (size_t)smax * sizeof(C);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_gal_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (int dir = 0; dir < 2; ++dir) {
    for (int jj = 0; jj < a.nblk - dir; ++jj) {
      const int j = dir ? a.nblk - 2 - jj : jj;
      const int Sj = (gal_row_hi(j, a.q) - gal_row_lo(j, a.q) + 1) * a.mc;
      const dim3 grid((unsigned)((Sj + 7) / 8), a.nrhs);  // 8 warps, one row each
      k_gal_step<T><<<grid, 256, (size_t)Sj * sizeof(C), s>>>(a, j, dir);
    }
  }
  return cudaGetLastError();
}

template cudaError_t launch_gal_apply<double>(const GalArgs<double>&, cudaStream_t);
template cudaError_t launch_gal_apply<float>(const GalArgs<float>&, cudaStream_t);
template cudaError_t launch_gal_solve<double>(const GalArgs<double>&, cudaStream_t);
template cudaError_t launch_gal_solve<float>(const GalArgs<float>&, cudaStream_t);

}  // namespace th
