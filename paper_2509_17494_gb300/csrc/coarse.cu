// K8: direct solve of the coarse QSFEM system A_q u_c = r_c (Algorithm 1,
// "solve u_c from A_c u_c = r_c"; Section 3.3 for A_q).
//
// Ordered by coarse grid rows, A_q is block tridiagonal: blocks D_j on the
// diagonal, C_j = A[row j, row j+1] above and B_j = C_{j-1}^T below (A_q is
// complex symmetric).  The FP64 set-up stores G_j = S_j^{-1} for the block
// Schur complements S_0 = D_0, S_j = D_j - B_j G_{j-1} C_{j-1}.  The solve is
//   forward   z_0 = G_0 r_0,  z_j = G_j (r_j - B_j z_{j-1}),
//   backward  x_{mc-1} = z_{mc-1},  x_j = z_j - G_j C_j x_{j+1}.
// One thread-block cluster per right-hand side runs the 2 mc - 1 dependent
// steps.  CTA c of the cluster owns rows [c rpc, (c+1) rpc) of every block
// vector; each step gathers the previous block vector from the cluster's
// shared memories (distributed shared memory), forms the tridiagonal
// product locally, computes its rows of the dense product with a warp per
// row, and meets the other CTAs at one hardware cluster barrier.  Slices are
// double-buffered so one barrier per step is enough.  There are no spin
// waits: every CTA executes the same number of barriers.
#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace th {

template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

template <typename T>
__global__ void __launch_bounds__(512) k_coarse_solve(const CoarseSolveArgs<T> a) {
  using C = typename Cx<T>::t;
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  const int csz = (int)cl.num_blocks();
  const int rhs = blockIdx.x / csz;
  const int mc = a.mc, rpc = a.rpc;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* own = reinterpret_cast<C*>(smraw);  // [2][rpc]
  C* full = own + 2 * rpc;               // [mc]
  C* tv = full + mc;                     // [mc]
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
  const int row0 = crank * rpc;
  const int nrow = max(0, min(rpc, mc - row0));
  const C* b = a.rhs + (size_t)rhs * a.Nc;
  C* z = a.z + (size_t)rhs * a.Nc;
  C* x = a.x + (size_t)rhs * a.Nc;

  auto gather = [&](int buf) {
    for (int k = tid; k < mc; k += nth) {
      const int rk = k / rpc, lk = k - rk * rpc;
      const C* remote = cl.map_shared_rank(own + buf * rpc, rk);
      full[k] = remote[lk];
    }
  };
  auto rowdot = [&](const C* Gj, int k) {
    const C* grow = Gj + (size_t)k * mc;
    T sr = 0, si = 0;
    for (int c = lane; c < mc; c += 32) {
      const C g = grow[c];
      const C t = tv[c];
      sr = fmadd(g.x, t.x, sr);
      sr = fmadd(-g.y, t.y, sr);
      si = fmadd(g.x, t.y, si);
      si = fmadd(g.y, t.x, si);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    C r;
    r.x = sr;
    r.y = si;
    return r;
  };

  // ---------------------------------------------------------------- forward
  for (int j = 0; j < mc; ++j) {
    if (j > 0) {
      gather((j - 1) & 1);
      __syncthreads();
      const size_t o = (size_t)(j - 1) * mc;
      for (int k = tid; k < mc; k += nth) {
        C t = b[(size_t)j * mc + k];
        C v = cmulc(a.cd[o + k], full[k]);
        if (k > 0) { const C w = cmulc(a.cu[o + k - 1], full[k - 1]); v.x += w.x; v.y += w.y; }
        if (k + 1 < mc) { const C w = cmulc(a.cl[o + k + 1], full[k + 1]); v.x += w.x; v.y += w.y; }
        t.x -= v.x;
        t.y -= v.y;
        tv[k] = t;
      }
    } else {
      for (int k = tid; k < mc; k += nth) tv[k] = b[k];
    }
    __syncthreads();
    const C* Gj = a.G + (size_t)j * mc * mc;
    for (int rr = warp; rr < nrow; rr += nwarps) {
      const C r = rowdot(Gj, row0 + rr);
      if (lane == 0) {
        own[(j & 1) * rpc + rr] = r;
        z[(size_t)j * mc + row0 + rr] = r;
      }
    }
    cl.sync();
  }
  // --------------------------------------------------------------- backward
  for (int rr = warp; rr < nrow; rr += nwarps)
    if (lane == 0) x[(size_t)(mc - 1) * mc + row0 + rr] = own[((mc - 1) & 1) * rpc + rr];
  for (int j = mc - 2; j >= 0; --j) {
    gather((j + 1) & 1);
    __syncthreads();
    const size_t o = (size_t)j * mc;
    for (int k = tid; k < mc; k += nth) {
      C v = cmulc(a.cd[o + k], full[k]);
      if (k > 0) { const C w = cmulc(a.cl[o + k], full[k - 1]); v.x += w.x; v.y += w.y; }
      if (k + 1 < mc) { const C w = cmulc(a.cu[o + k], full[k + 1]); v.x += w.x; v.y += w.y; }
      tv[k] = v;
    }
    __syncthreads();
    const C* Gj = a.G + (size_t)j * mc * mc;
    for (int rr = warp; rr < nrow; rr += nwarps) {
      const C r = rowdot(Gj, row0 + rr);
      if (lane == 0) {
        const C zz = z[(size_t)j * mc + row0 + rr];
        C xv;
        xv.x = zz.x - r.x;
        xv.y = zz.y - r.y;
        own[(j & 1) * rpc + rr] = xv;
        x[(size_t)j * mc + row0 + rr] = xv;
      }
    }
    cl.sync();
  }
}

template <typename T>
cudaError_t launch_coarse_solve(const CoarseSolveArgs<T>& a, int nrhs, int cluster, cudaStream_t s) {
  using C = typename Cx<T>::t;
  const size_t smem = sizeof(C) * (size_t)(2 * a.rpc + 2 * a.mc);
  cudaError_t e = cudaFuncSetAttribute(k_coarse_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(k_coarse_solve<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster * nrhs, 1, 1);
  cfg.blockDim = dim3(512, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_coarse_solve<T>, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template cudaError_t launch_coarse_solve<double>(const CoarseSolveArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_coarse_solve<float>(const CoarseSolveArgs<float>&, int, int, cudaStream_t);

}  // namespace th
