// K8: partitioned direct solve of the coarse QSFEM system A_q u_c = r_c
// (Algorithm 1, "solve u_c from A_c u_c = r_c"; A_q of Section 3.3).
//
// A_q ordered by coarse grid rows is block tridiagonal.  The rows are split
// into P chunks separated by P - 1 separator rows (set-up: coarse_partition).
// The solve runs in three launches:
//   1. k_chunk_sweep: one thread-block cluster per (chunk, rhs) runs the block
//      LU sweep of its chunk alone, y = A_cc^{-1} b_c, writing y into the
//      output.  The chunks run concurrently, so the dependent chain is the
//      chunk length (about sqrt(m_c)) instead of m_c.
//   2. k_reduced_rhs + k_reduced_gemv: the separator rows satisfy a small
//      dense system (P - 1 block rows); its right-hand side is formed from y
//      and its FP64-set-up explicit inverse is applied as one row-parallel
//      GEMV, writing the separator values into the output.
//   3. k_spike_correct: every chunk row gets x_j = y_j - L_j x_left - R_j x_right
//      (dense spike blocks, all rows in parallel).
// Inside a cluster, CTA c owns rows [c rpc, (c+1) rpc) of every block vector.
// After computing its rows of a block vector a CTA writes them into every
// CTA's shared memory of the cluster (distributed shared memory), then all
// meet at one hardware cluster barrier; the next block's rows of G are
// prefetched with cp.async into a double buffer one step ahead.  There are no
// spin waits: every CTA of a cluster executes the same number of barriers.
#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace th {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename C>
__device__ __forceinline__ void cmac(C& acc, C a, C b) {
  acc.x += a.x * b.x - a.y * b.y;
  acc.y += a.x * b.y + a.y * b.x;
}

template <typename T>
__device__ __forceinline__ typename Cx<T>::t warp_sum(typename Cx<T>::t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// async copy of one complex value (8 or 16 bytes)
template <typename C>
__device__ __forceinline__ void cp_async_elem(C* smem, const C* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(C) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  }
}

// ------------------------------------------------------------- chunk sweep
// Step q (0 <= q < 2L - 1) handles block row j = block_of(q): forward
// z_j = G_j (b_j - C_{j-1}^T z_{j-1}) for q < L, backward
// y_j = z_j - G_j C_j y_{j+1} after.  Everything a step reads from global
// memory (its rows of G_j, the right-hand-side row b_j and the three
// coefficient rows of the tridiagonal coupling) is copied into shared memory
// by cp.async two steps ahead; results stay in shared memory until the loop
// ends, so no global access waits at the cluster barriers.
template <typename T, bool PREFETCH>
__global__ void __launch_bounds__(512, 1) k_chunk_sweep(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank(), csz = (int)cl.num_blocks();
  const int cid = blockIdx.x / csz;
  const int chunk = cid % a.P, rhs = cid / a.P;
  const int mc = a.mc, mcp = a.mcp, rpc = a.rpc;
  const int A = a.ca[chunk], L = a.cb[chunk] - A + 1;
  const int nsteps = 2 * L - 1;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
  const int row0 = crank * rpc, nrow = max(0, min(rpc, mc - row0));
  extern __shared__ __align__(16) unsigned char smraw[];
  C* gbuf = reinterpret_cast<C*>(smraw);                    // [2][rpc * mcp] (PREFETCH)
  C* ops = gbuf + (PREFETCH ? (size_t)2 * rpc * mcp : 0);   // [2][4][mc]: b, o0, o1, o2
  C* full = ops + (size_t)8 * mc;                           // [2][mc]
  C* tv = full + 2 * mc;                                    // [mc]
  C* zs = tv + mc;                                          // [Lmax][rpc]: z, then y
  const C* b = a.b + (size_t)rhs * a.Nc;
  C* x = a.x + (size_t)rhs * a.Nc;
  auto block_of = [&](int q) { return q < L ? A + q : A + (2 * L - 2 - q); };
  auto prefetch = [&](int q, int buf) {
    if (q < nsteps) {
      const int j = block_of(q);
      if (PREFETCH && nrow > 0) {
        const char* src = reinterpret_cast<const char*>(a.G + ((size_t)j * mc + row0) * mcp);
        char* dst = reinterpret_cast<char*>(gbuf + (size_t)buf * rpc * mcp);
        const int units = (int)((size_t)nrow * mcp * sizeof(C) / 16);
        for (int u = tid; u < units; u += nth) cp_async16(dst + (size_t)u * 16, src + (size_t)u * 16);
      }
      C* o = ops + (size_t)buf * 4 * mc;
      // forward: b_j and C_{j-1} rows (cd, cu, cl); backward: C_j rows (cd, cl, cu)
      const bool f = q < L;
      const size_t oc = (size_t)(f ? j - 1 : j) * mc;
      const C* r1 = f ? a.cu : a.cl;
      const C* r2 = f ? a.cl : a.cu;
      for (int k = tid; k < mc; k += nth) {
        if (f) cp_async_elem(o + k, b + (size_t)j * mc + k);
        if (!f || q > 0) {
          cp_async_elem(o + mc + k, a.cd + oc + k);
          cp_async_elem(o + 2 * mc + k, r1 + oc + k);
          cp_async_elem(o + 3 * mc + k, r2 + oc + k);
        }
      }
    }
    cp_async_commit();
  };
  prefetch(0, 0);
  prefetch(1, 1);
  for (int q = 0; q < nsteps; ++q) {
    const bool fwd = q < L;
    const int j = block_of(q);
    const C* prev = full + ((q - 1) & 1) * mc;
    const C* o = ops + (size_t)(q & 1) * 4 * mc;
    cp_async_wait<1>();
    __syncthreads();
    for (int k = tid; k < mc; k += nth) {
      C v;
      v.x = 0;
      v.y = 0;
      if (!fwd || q > 0) {
        cmac(v, o[mc + k], prev[k]);
        if (fwd) {  // C_{j-1}^T: cu[k-1] p[k-1] + cl[k+1] p[k+1]
          if (k > 0) cmac(v, o[2 * mc + k - 1], prev[k - 1]);
          if (k + 1 < mc) cmac(v, o[3 * mc + k + 1], prev[k + 1]);
        } else {    // C_j: cl[k] p[k-1] + cu[k] p[k+1]
          if (k > 0) cmac(v, o[2 * mc + k], prev[k - 1]);
          if (k + 1 < mc) cmac(v, o[3 * mc + k], prev[k + 1]);
        }
      }
      if (fwd) {
        C t = o[k];
        t.x -= v.x;
        t.y -= v.y;
        tv[k] = t;
      } else {
        tv[k] = v;
      }
    }
    __syncthreads();
    const C* Gr = PREFETCH ? gbuf + (size_t)(q & 1) * rpc * mcp : a.G + ((size_t)j * mc + row0) * mcp;
    C* dst = full + (q & 1) * mc;
    for (int rr = warp; rr < nrow; rr += nwarps) {
      const C* g = Gr + (size_t)rr * mcp;
      C acc;
      acc.x = 0;
      acc.y = 0;
      for (int c = lane; c < mc; c += 32) cmac(acc, g[c], tv[c]);
      acc = warp_sum<T>(acc);
      C val = acc;
      const size_t zi = (size_t)(j - A) * rpc + rr;
      if (!fwd) {
        const C z = zs[zi];
        val.x = z.x - acc.x;
        val.y = z.y - acc.y;
      }
      __syncwarp();
      if (lane == 0) zs[zi] = val;  // z_j forward, y_j backward (y_{A+L-1} = z_{A+L-1})
      if (lane < csz) {
        C* remote = cl.map_shared_rank(dst, lane);
        remote[row0 + rr] = val;
      }
    }
    cluster_arrive_release();
    cluster_wait_acquire();
    prefetch(q + 2, q & 1);
  }
  cp_async_wait<0>();
  __syncthreads();
  for (int i = tid; i < L * nrow; i += nth) {
    const int jj = i / nrow, rr = i - jj * nrow;
    x[(size_t)(A + jj) * mc + row0 + rr] = zs[(size_t)jj * rpc + rr];
  }
}

// ------------------------------------------------------------- reduced system
// rhat_k = b_s - C_{s-1}^T y_{s-1} - C_s y_{s+1} for every separator row s = sep[k]
template <typename T>
__global__ void __launch_bounds__(256) k_reduced_rhs(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nred) return;
  const int mc = a.mc;
  const int k = i / mc, e = i - k * mc;
  const int s = a.sep[k];
  const C* b = a.b + (size_t)blockIdx.y * a.Nc;
  const C* x = a.x + (size_t)blockIdx.y * a.Nc;
  const C* ym = x + (size_t)(s - 1) * mc;
  const C* yp = x + (size_t)(s + 1) * mc;
  const size_t om = (size_t)(s - 1) * mc, os = (size_t)s * mc;
  C t = b[os + e];
  C v;
  v.x = 0;
  v.y = 0;
  cmac(v, a.cd[om + e], ym[e]);
  if (e > 0) cmac(v, a.cu[om + e - 1], ym[e - 1]);
  if (e + 1 < mc) cmac(v, a.cl[om + e + 1], ym[e + 1]);
  cmac(v, a.cd[os + e], yp[e]);
  if (e > 0) cmac(v, a.cl[os + e], yp[e - 1]);
  if (e + 1 < mc) cmac(v, a.cu[os + e], yp[e + 1]);
  t.x -= v.x;
  t.y -= v.y;
  a.rhat[(size_t)blockIdx.y * a.nred + i] = t;
}

// xhat = Sinv rhat, one warp per row, written into the separator rows of x
template <typename T>
__global__ void __launch_bounds__(256) k_reduced_gemv(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  const int lane = threadIdx.x & 31;
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= a.nred) return;
  const C* srow = a.Sinv + (size_t)row * a.nred;
  const C* r = a.rhat + (size_t)blockIdx.y * a.nred;
  C acc;
  acc.x = 0;
  acc.y = 0;
  for (int c = lane; c < a.nred; c += 32) cmac(acc, srow[c], r[c]);
  acc = warp_sum<T>(acc);
  if (lane == 0) {
    const int k = (int)(row / a.mc), e = (int)(row - (long long)k * a.mc);
    a.x[(size_t)blockIdx.y * a.Nc + (size_t)a.sep[k] * a.mc + e] = acc;
  }
}

// ------------------------------------------------------------- spike correction
template <typename T>
__global__ void __launch_bounds__(256) k_spike_correct(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  const int mc = a.mc, mcp = a.mcp;
  const int lane = threadIdx.x & 31;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nrows = (long long)mc * mc;
  if (wid >= nrows) return;
  const int j = (int)(wid / mc), e = (int)(wid - (long long)j * mc);
  const int c = a.chunk_of[j];
  if (c < 0) return;  // separator row
  C* x = a.x + (size_t)blockIdx.y * a.Nc;
  const C* row = a.LR + ((size_t)j * mc + e) * 2 * mcp;
  C acc;
  acc.x = 0;
  acc.y = 0;
  if (c > 0) {
    const C* xl = x + (size_t)a.sep[c - 1] * mc;
    for (int r = lane; r < mc; r += 32) cmac(acc, row[r], xl[r]);
  }
  if (c < a.P - 1) {
    const C* xr = x + (size_t)a.sep[c] * mc;
    for (int r = lane; r < mc; r += 32) cmac(acc, row[mcp + r], xr[r]);
  }
  acc = warp_sum<T>(acc);
  if (lane == 0) {
    C v = x[(size_t)j * mc + e];
    v.x -= acc.x;
    v.y -= acc.y;
    x[(size_t)j * mc + e] = v;
  }
}

// ------------------------------------------------------------- launcher
template <typename T>
size_t chunk_sweep_smem(const CoarsePartArgs<T>& a, bool prefetch) {
  using C = typename Cx<T>::t;
  size_t s = sizeof(C) * ((size_t)11 * a.mc + (size_t)a.Lmax * a.rpc);
  if (prefetch) s += sizeof(C) * (size_t)2 * a.rpc * a.mcp;
  return s;
}

template <typename K, typename Args>
static cudaError_t launch_cluster(K kern, const Args& a, int grid, int cluster, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
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
  e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_part(const CoarsePartArgs<T>& a, int nrhs, int cluster, cudaStream_t s) {
  const bool pf = chunk_sweep_smem(a, true) <= 220 * 1024;
  const size_t sm1 = chunk_sweep_smem(a, pf);
  cudaError_t e = pf ? launch_cluster(k_chunk_sweep<T, true>, a, cluster * a.P * nrhs, cluster, sm1, s)
                     : launch_cluster(k_chunk_sweep<T, false>, a, cluster * a.P * nrhs, cluster, sm1, s);
  if (e != cudaSuccess || a.P < 2) return e;
  {
    dim3 g1((unsigned)((a.nred + 255) / 256), nrhs);
    k_reduced_rhs<T><<<g1, 256, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g2((unsigned)(((long long)a.nred * 32 + 255) / 256), nrhs);
    k_reduced_gemv<T><<<g2, 256, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const long long warps = (long long)a.mc * a.mc;
  dim3 grid((unsigned)((warps * 32 + 255) / 256), nrhs);
  k_spike_correct<T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_coarse_part<double>(const CoarsePartArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_coarse_part<float>(const CoarsePartArgs<float>&, int, int, cudaStream_t);

}  // namespace th
