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
//   2. k_reduced_rhs + k_coarse_tsgemm<MODE 0>: the separator rows satisfy a
//      small dense system (P - 1 block rows); its right-hand side is formed
//      from y and its FP64-set-up explicit inverse is applied as one
//      row-parallel product, writing the separator values into the output.
//   3. k_coarse_tsgemm<MODE 1>: every chunk row gets
//      x_j = y_j - L_j x_left - R_j x_right (dense spike blocks, all rows in
//      parallel).
// With several right-hand sides, k_chunk_sweep_mr and the NB-column
// k_coarse_tsgemm take tiles of them (below).
// Inside a cluster, CTA c owns rows [c rpc, (c+1) rpc) of every block vector.
// After computing its rows of a block vector a CTA writes them into every
// CTA's shared memory of the cluster (distributed shared memory), then all
// meet at one hardware cluster barrier; the next block's rows of G are
// prefetched with cp.async into a double buffer one step ahead.  There are no
// spin waits: every CTA of a cluster executes the same number of barriers.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

#include "kernels.h"
#include "launch.cuh"
#include "ptx.cuh"

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
  cmadd(acc, a, b);
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

// Variant for m_c <= 256 with at most 32 rows per CTA: 32 warps, one row each,
// and two barriers per block step instead of three: the vector G_j multiplies
// is formed cooperatively (one entry per thread) and one CTA barrier separates
// it from the products; each thread waits for its own prefetch copies before
// the cluster barrier that ends the step, which then also makes every copy and
// every pushed row visible to the next step.
template <typename T, bool PREFETCH>
__global__ void __launch_bounds__(1024, 1) k_chunk_sweep1(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  constexpr int NI = 8;
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank(), csz = (int)cl.num_blocks();
  const int cid = blockIdx.x / csz;
  const int chunk = cid % a.P, rhs = cid / a.P;
  const int mc = a.mc, mcp = a.mcp, rpc = a.rpc;
  const int A = a.ca[chunk], L = a.cb[chunk] - A + 1;
  const int nsteps = 2 * L - 1;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = crank * rpc, nrow = max(0, min(rpc, mc - row0));
  extern __shared__ __align__(16) unsigned char smraw[];
  C* gbuf = reinterpret_cast<C*>(smraw);                    // [2][rpc * mcp] (PREFETCH)
  C* ops = gbuf + (PREFETCH ? (size_t)2 * rpc * mcp : 0);   // [2][4][mc]: b, o0, o1, o2
  C* full = ops + (size_t)8 * mc;                           // [2][mc]
  C* tvs = full + 2 * mc;                                   // [mc]
  C* zs = tvs + mc;                                         // [Lmax][rpc]: z, then y
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
  cp_async_wait<1>();
  __syncthreads();
  for (int q = 0; q < nsteps; ++q) {
    const bool fwd = q < L;
    const int j = block_of(q);
    const C* prev = full + ((q - 1) & 1) * mc;
    const C* o = ops + (size_t)(q & 1) * 4 * mc;
    // the vector: forward b_j - C_{j-1}^T prev, backward C_j prev (one entry per thread)
    for (int k = tid; k < mc; k += nth) {
      C v;
      v.x = 0;
      v.y = 0;
      if (!fwd || q > 0) {
        cmac(v, o[mc + k], prev[k]);
        if (fwd) {
          if (k > 0) cmac(v, o[2 * mc + k - 1], prev[k - 1]);
          if (k + 1 < mc) cmac(v, o[3 * mc + k + 1], prev[k + 1]);
        } else {
          if (k > 0) cmac(v, o[2 * mc + k], prev[k - 1]);
          if (k + 1 < mc) cmac(v, o[3 * mc + k], prev[k + 1]);
        }
      }
      if (fwd) {
        const C bk = o[k];
        v.x = bk.x - v.x;
        v.y = bk.y - v.y;
      }
      tvs[k] = v;
    }
    __syncthreads();
    C tv[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int k = lane + 32 * i;
      if (k < mc) {
        tv[i] = tvs[k];
      } else {
        tv[i].x = 0;
        tv[i].y = 0;
      }
    }
    const int rr = warp;
    if (rr < nrow) {
      const C* g = PREFETCH ? gbuf + (size_t)(q & 1) * rpc * mcp + (size_t)rr * mcp
                            : a.G + ((size_t)j * mc + row0 + rr) * mcp;
      C acc;
      acc.x = 0;
      acc.y = 0;
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int k = lane + 32 * i;
        if (k < mc) cmac(acc, g[k], tv[i]);
      }
      acc = warp_sum<T>(acc);
      const size_t zi = (size_t)(j - A) * rpc + rr;
      C val = acc;
      if (!fwd) {
        const C z = zs[zi];
        val.x = z.x - acc.x;
        val.y = z.y - acc.y;
      }
      if (lane == 0) zs[zi] = val;
      if (lane < csz) {
        C* remote = cl.map_shared_rank(full + (q & 1) * mc, lane);
        remote[row0 + rr] = val;
      }
    }
    cp_async_wait<0>();
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

// Variant 2: the rows a CTA computes reach the other CTAs of the cluster by
// st.async stores that complete transactions on the receivers' mbarriers
// (one per exchange slot), so a block step ends without a cluster barrier:
// each CTA waits only for the mc values it needs.  The G rows of the coming
// steps are prefetched into a ring of three buffers.  Slot reuse is safe
// without further synchronisation: a CTA writes step q's rows into slot q&1
// only after it received every row of step q-1, which every receiver sends
// after it finished reading slot q&1 (its step q-1 input).  Waits are bounded;
// on a timeout the CTA flags the error and finishes without waiting.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned mapa_u32(unsigned addr, int rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_async_c(unsigned raddr, float2 v, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];\n"
               ::"r"(raddr), "f"(v.x), "f"(v.y), "r"(rbar) : "memory");
}
__device__ __forceinline__ void st_async_c(unsigned raddr, double2 v, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];\n"
               ::"r"(raddr), "d"(v.x), "d"(v.y), "r"(rbar) : "memory");
}
template <typename T>
__global__ void __launch_bounds__(1024, 1) k_chunk_sweep2(const CoarsePartArgs<T> a, int* err) {
  using C = typename Cx<T>::t;
  constexpr int NI = 8;
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank(), csz = (int)cl.num_blocks();
  const int cid = blockIdx.x / csz;
  const int chunk = cid % a.P, rhs = cid / a.P;
  const int mc = a.mc, mcp = a.mcp, rpc = a.rpc;
  const int A = a.ca[chunk], L = a.cb[chunk] - A + 1;
  const int nsteps = 2 * L - 1;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = crank * rpc, nrow = max(0, min(rpc, mc - row0));
  extern __shared__ __align__(16) unsigned char smraw[];
  uint64_t* fbar = reinterpret_cast<uint64_t*>(smraw);          // [2] exchange-slot barriers
  C* gbuf = reinterpret_cast<C*>(smraw + 16);                   // [3][rpc * mcp]
  C* ops = gbuf + (size_t)3 * rpc * mcp;                        // [2][4][mc]: b, o0, o1, o2
  C* full = ops + (size_t)8 * mc;                               // [2][mc]
  C* tvs = full + 2 * mc;                                       // [mc]
  C* zs = tvs + mc;                                             // [Lmax][rpc]: z, then y
  __shared__ int failed;
  const C* b = a.b + (size_t)rhs * a.Nc;
  C* x = a.x + (size_t)rhs * a.Nc;
  const unsigned slot_bytes = (unsigned)(mc * sizeof(C));
  auto block_of = [&](int q) { return q < L ? A + q : A + (2 * L - 2 - q); };
  // The G rows are copied by the warps that have no row of their own (warps
  // rpc .. 31) when there are such warps, so the row warps start their
  // products right after the step's barrier; otherwise by every thread.
  const int cw0 = rpc < nth / 32 ? rpc : 0;
  auto prefetch = [&](int q) {
    if (q < nsteps) {
      const int j = block_of(q);
      if (nrow > 0 && warp >= cw0) {
        const char* src = reinterpret_cast<const char*>(a.G + ((size_t)j * mc + row0) * mcp);
        char* dst = reinterpret_cast<char*>(gbuf + (size_t)(q % 3) * rpc * mcp);
        const int units = (int)((size_t)nrow * mcp * sizeof(C) / 16);
        for (int u = tid - cw0 * 32; u < units; u += nth - cw0 * 32)
          cp_async16(dst + (size_t)u * 16, src + (size_t)u * 16);
      }
      // operands staged per entry k by the thread that later uses them, so the
      // vector needs no CTA barrier after the copies: b_j[k], the diagonal
      // coupling and the two off-diagonal ones, each at index k
      C* o = ops + (size_t)(q & 1) * 4 * mc;
      const bool f = q < L;
      const size_t oc = (size_t)(f ? j - 1 : j) * mc;
      for (int k = tid; k < mc; k += nth) {
        if (f) cp_async_elem(o + k, b + (size_t)j * mc + k);
        if (!f || q > 0) {
          cp_async_elem(o + mc + k, a.cd + oc + k);
          if (f) {  // C_{j-1}^T: cu[k-1] p[k-1] + cl[k+1] p[k+1]
            if (k > 0) cp_async_elem(o + 2 * mc + k, a.cu + oc + k - 1);
            if (k + 1 < mc) cp_async_elem(o + 3 * mc + k, a.cl + oc + k + 1);
          } else {  // C_j: cl[k] p[k-1] + cu[k] p[k+1]
            if (k > 0) cp_async_elem(o + 2 * mc + k, a.cl + oc + k);
            if (k + 1 < mc) cp_async_elem(o + 3 * mc + k, a.cu + oc + k);
          }
        }
      }
    }
    cp_async_commit();
  };
  // rows are sent at steps 0 .. nsteps - 2 (the last step's rows stay local)
  const int nsend = nsteps - 1;
  const int lim = ptx::wait_limit(err, 1 << 20);
  if (lim == 0) {  // waits disabled (the same for every CTA of the cluster): no barrier, copy or store
    if (tid == 0 && crank == 0) atomicExch(err, 1);
    return;
  }
  if (tid == 0) {
    failed = 0;
    ptx::mbar_init(fbar + 0, 1);
    ptx::mbar_init(fbar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (nsend > 0) ptx::mbar_arrive_expect_tx(fbar + 0, slot_bytes);
    if (nsend > 1) ptx::mbar_arrive_expect_tx(fbar + 1, slot_bytes);
  }
  // every barrier is initialised before any CTA of the cluster can send to it
  cluster_arrive_release();
  cluster_wait_acquire();
  ptx::grid_dep_wait();  // b is the previous kernel's output
  ptx::grid_dep_launch();
  prefetch(0);
  prefetch(1);
  for (int q = 0; q < nsteps; ++q) {
    const bool fwd = q < L;
    const int j = block_of(q);
    if (q > 0) {  // step q-1's rows, from every CTA of the cluster
      uint64_t* bar = fbar + ((q - 1) & 1);
      const unsigned par = (unsigned)(((q - 1) >> 1) & 1);
      if (!failed) {
        bool ok = false;
        for (int it = 0; it < lim && !ok; ++it) ok = ptx::mbar_try_wait_cluster(bar, par);
        if (!ok) failed = 1;
      }
    }
    cp_async_wait<1>();  // this thread's copies of this step (the next step's may be in flight)
    const C* prev = full + ((q - 1) & 1) * mc;
    const C* o = ops + (size_t)(q & 1) * 4 * mc;
    for (int k = tid; k < mc; k += nth) {
      C v;
      v.x = 0;
      v.y = 0;
      if (!fwd || q > 0) {
        cmac(v, o[mc + k], prev[k]);
        if (k > 0) cmac(v, o[2 * mc + k], prev[k - 1]);
        if (k + 1 < mc) cmac(v, o[3 * mc + k], prev[k + 1]);
      }
      if (fwd) {
        const C bk = o[k];
        v.x = bk.x - v.x;
        v.y = bk.y - v.y;
      }
      tvs[k] = v;
    }
    __syncthreads();  // tvs and the G rows are visible; every thread is past its wait
    // the slot just consumed takes the rows of step q + 1
    if (tid == 0 && q > 0 && q + 1 <= nsend - 1 && !failed) ptx::mbar_arrive_expect_tx(fbar + ((q - 1) & 1), slot_bytes);
    // step q + 2's copies: G into buffer (q + 2) % 3 (last read at step q - 1)
    prefetch(q + 2);
    const int rr = warp;
    if (rr < nrow) {
      C tv[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int k = lane + 32 * i;
        if (k < mc) {
          tv[i] = tvs[k];
        } else {
          tv[i].x = 0;
          tv[i].y = 0;
        }
      }
      const C* g = gbuf + (size_t)(q % 3) * rpc * mcp + (size_t)rr * mcp;
      C acc;
      acc.x = 0;
      acc.y = 0;
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int k = lane + 32 * i;
        if (k < mc) cmac(acc, g[k], tv[i]);
      }
      acc = warp_sum<T>(acc);
      const size_t zi = (size_t)(j - A) * rpc + rr;
      C val = acc;
      if (!fwd) {
        const C z = zs[zi];
        val.x = z.x - acc.x;
        val.y = z.y - acc.y;
      }
      if (lane == 0) zs[zi] = val;
      if (q < nsend && lane < csz) {
        const unsigned slot = smem_u32(full + (q & 1) * mc + row0 + rr);
        st_async_c(mapa_u32(slot, lane), val, mapa_u32(smem_u32(fbar + (q & 1)), lane));
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  for (int i = tid; i < L * nrow; i += nth) {
    const int jj = i / nrow, rr = i - jj * nrow;
    x[(size_t)(A + jj) * mc + row0 + rr] = zs[(size_t)jj * rpc + rr];
  }
  if (tid == 0 && failed) atomicExch(err, 1);
  // no CTA leaves while another may still store into its shared memory
  cluster_arrive_release();
  cluster_wait_acquire();
}

// ------------------------------------------------------------- reduced system
// rhat_k = b_s - C_{s-1}^T y_{s-1} - C_s y_{s+1} for every separator row s = sep[k]
template <typename T>
__global__ void __launch_bounds__(256) k_reduced_rhs(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  ptx::grid_dep_wait();  // launched with a programmatic dependency inside the cycle
  ptx::grid_dep_launch();
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
  if (a.rst) {  // split-BF16 operand chunks of the tensor-core separator product (coarse_umma.cu)
    const int rhs = blockIdx.y, n = rhs & 63;
    __nv_bfloat16* st =
        reinterpret_cast<__nv_bfloat16*>(a.rst + ((size_t)(rhs >> 6) * a.nkc_s + (i >> 5)) * (4 * 64 * 32 * 2));
    const int off = umma_off32(n, i & 31);
    const float vr = (float)t.x, vi = (float)t.y;
    const __nv_bfloat16 hr = __float2bfloat16_rn(vr), hi = __float2bfloat16_rn(vi);
    st[off] = hr;
    st[64 * 32 + off] = hi;
    st[2 * 64 * 32 + off] = __float2bfloat16_rn(vr - __bfloat162float(hr));
    st[3 * 64 * 32 + off] = __float2bfloat16_rn(vi - __bfloat162float(hi));
    return;
  }
  a.rhat[(size_t)blockIdx.y * a.nred + i] = t;
}

// ------------------------------------------------------------- many right-hand sides
// The same three stages for a tile of NB right-hand sides per cluster / warp:
// every block of G, of the spikes and of the reduced inverse is read once per
// tile instead of once per right-hand side, and the tile index varies fastest
// in the grid so that the clusters running at the same time read the same
// blocks (through L2).  The tile's vectors are stored [row][rhs] in shared
// memory.  Each CTA splits the columns of its G_j rows over its warps; a lane
// owns one row and NB accumulators, reads its row's entry of the transposed
// G_j (consecutive across lanes) and the column's NB vector entries (the same
// address for the whole warp); the warps' partial sums are then added in a
// fixed order, so the result is bitwise deterministic.
template <typename T, int NB, bool PREFETCH>
__global__ void __launch_bounds__(512, 1) k_chunk_sweep_mr(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  constexpr int NW = 16;  // warps per CTA
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank(), csz = (int)cl.num_blocks();
  const int cid = blockIdx.x / csz;
  const int ntiles = (a.nrhs + NB - 1) / NB;
  const int tile = cid % ntiles, chunk = cid / ntiles;
  const int r0 = tile * NB, nb = min(NB, a.nrhs - r0);
  const int mc = a.mc, rpc = a.rpcm, mcr = a.mcr;
  const int A = a.ca[chunk], L = a.cb[chunk] - A + 1;
  const int nsteps = 2 * L - 1;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = crank * rpc, nrow = max(0, min(rpc, mc - row0));
  const int cs = (mc + NW - 1) / NW, c0 = min(mc, warp * cs), c1 = min(mc, c0 + cs);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* gbuf = reinterpret_cast<C*>(smraw);                      // [2][mc][rpc] (PREFETCH)
  C* bops = gbuf + (PREFETCH ? (size_t)2 * mc * rpc : 0);     // [2][mc][NB]
  C* cops = bops + (size_t)2 * mc * NB;                       // [2][3][mc]
  C* full = cops + (size_t)6 * mc;                            // [2][mc][NB]
  C* tv = full + (size_t)2 * mc * NB;                         // [mc][NB]
  C* red = tv + (size_t)mc * NB;                              // [NW][rpc][NB + 1]
  C* zs = red + (size_t)NW * rpc * (NB + 1);                  // [Lmax][rpc][NB]: z, then y
  auto block_of = [&](int q) { return q < L ? A + q : A + (2 * L - 2 - q); };
  auto prefetch = [&](int q, int buf) {
    if (q < nsteps) {
      const int j = block_of(q);
      if (PREFETCH && nrow > 0) {
        const char* src = reinterpret_cast<const char*>(a.Gt + (size_t)j * mc * mcr + row0);
        char* dst = reinterpret_cast<char*>(gbuf + (size_t)buf * mc * rpc);
        const int units = (int)(rpc * sizeof(C) / 16);  // per column: this CTA's rows (padded)
        for (int u = tid; u < mc * units; u += nth) {
          const int c = u / units, w = u - c * units;
          cp_async16(dst + ((size_t)c * rpc * sizeof(C) + (size_t)w * 16),
                     src + ((size_t)c * mcr * sizeof(C) + (size_t)w * 16));
        }
      }
      const bool f = q < L;
      C* o = cops + (size_t)buf * 3 * mc;
      const size_t oc = (size_t)(f ? j - 1 : j) * mc;
      const C* r1 = f ? a.cu : a.cl;
      const C* r2 = f ? a.cl : a.cu;
      if (!f || q > 0) {
        for (int k = tid; k < mc; k += nth) {
          cp_async_elem(o + k, a.cd + oc + k);
          cp_async_elem(o + mc + k, r1 + oc + k);
          cp_async_elem(o + 2 * mc + k, r2 + oc + k);
        }
      }
      if (f) {  // b_j of the tile's right-hand sides (a ragged tile repeats its last one)
        C* bo = bops + (size_t)buf * mc * NB;
        for (int i = tid; i < NB * mc; i += nth) {
          const int r = i / mc, k = i - r * mc;
          const C* src = a.b + (size_t)(r0 + min(r, nb - 1)) * a.Nc + (size_t)j * mc + k;
          cp_async_elem(bo + (size_t)k * NB + r, src);
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
    const C* prev = full + (size_t)((q - 1) & 1) * mc * NB;
    const C* o = cops + (size_t)(q & 1) * 3 * mc;
    const C* bo = bops + (size_t)(q & 1) * mc * NB;
    cp_async_wait<1>();
    __syncthreads();
    for (int i = tid; i < mc * NB; i += nth) {
      const int k = i / NB;
      C v;
      v.x = 0;
      v.y = 0;
      if (!fwd || q > 0) {
        cmac(v, o[k], prev[i]);
        if (fwd) {  // C_{j-1}^T
          if (k > 0) cmac(v, o[mc + k - 1], prev[i - NB]);
          if (k + 1 < mc) cmac(v, o[2 * mc + k + 1], prev[i + NB]);
        } else {    // C_j
          if (k > 0) cmac(v, o[mc + k], prev[i - NB]);
          if (k + 1 < mc) cmac(v, o[2 * mc + k], prev[i + NB]);
        }
      }
      if (fwd) {
        C tt = bo[i];
        tt.x -= v.x;
        tt.y -= v.y;
        tv[i] = tt;
      } else {
        tv[i] = v;
      }
    }
    __syncthreads();
    // partial products over this warp's columns
    const C* Gs = PREFETCH ? gbuf + (size_t)(q & 1) * mc * rpc : nullptr;
    const C* Gg = a.Gt + (size_t)j * mc * mcr + row0;
    for (int rr = lane; rr < nrow; rr += 32) {
      C acc[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        acc[r].x = 0;
        acc[r].y = 0;
      }
#pragma unroll 4
      for (int c = c0; c < c1; ++c) {
        const C g = PREFETCH ? Gs[(size_t)c * rpc + rr] : Gg[(size_t)c * mcr + rr];
        const C* tc = tv + (size_t)c * NB;
#pragma unroll
        for (int r = 0; r < NB; ++r) cmac(acc[r], g, tc[r]);
      }
#pragma unroll
      for (int r = 0; r < NB; ++r) red[((size_t)warp * rpc + rr) * (NB + 1) + r] = acc[r];
    }
    __syncthreads();
    C* dst = full + (size_t)(q & 1) * mc * NB;
    for (int i = tid; i < nrow * NB; i += nth) {
      const int rr = i / NB, r = i - rr * NB;
      C s;
      s.x = 0;
      s.y = 0;
      for (int w = 0; w < NW; ++w) {
        if (w * cs >= mc) break;
        const C v = red[((size_t)w * rpc + rr) * (NB + 1) + r];
        s.x += v.x;
        s.y += v.y;
      }
      const size_t zi = ((size_t)(j - A) * rpc + rr) * NB + r;
      C val = s;
      if (!fwd) {
        const C z = zs[zi];
        val.x = z.x - s.x;
        val.y = z.y - s.y;
      }
      zs[zi] = val;  // z_j forward, y_j backward (y_{A+L-1} = z_{A+L-1})
      for (int d = 0; d < csz; ++d) {
        C* remote = cl.map_shared_rank(dst, d);
        remote[(size_t)(row0 + rr) * NB + r] = val;
      }
    }
    cluster_arrive_release();
    cluster_wait_acquire();
    prefetch(q + 2, q & 1);
  }
  cp_async_wait<0>();
  __syncthreads();
  for (int i = tid; i < nb * L * nrow; i += nth) {
    const int r = i / (L * nrow), rem = i - r * (L * nrow);
    const int jj = rem / nrow, rr = rem - jj * nrow;
    a.x[(size_t)(r0 + r) * a.Nc + (size_t)(A + jj) * mc + row0 + rr] = zs[((size_t)jj * rpc + rr) * NB + r];
  }
}

// ------------------------------------------------------------- wide tiles of right-hand sides
// The chunk sweep for a group of NBW right-hand sides per CTA (NBW from 8 to 16,
// the narrowest that keeps P x groups within one CTA per SM): one CTA per
// (chunk, group), no cluster.  A thread owns rows of the block (row rr for
// rr = tid, tid + blockDim, ...) and NBW accumulators; it streams its row's
// entries of the transposed G_j (consecutive across lanes, through L2: the
// CTAs of the other groups of the same chunk read the same G_j at about the
// same time) and reads the step's vector block T_j[c][0..NBW-1] from shared
// memory (the same address for the whole warp).  Per step
//   forward  (q < L):  T = b_j - C_{j-1}^T z_{j-1},  z_j = G_j T,
//   backward (q >= L): T = C_j y_{j+1},             y_j = z_j - G_j T,
// with z_j kept in the output x between the passes (x[j] = z_j, then y_j)
// and the previous step's block in shared memory.  Each G_j is read from
// HBM about once per sweep for all right-hand sides (the per-tile sweep
// above reads it once per tile), and the grid has P x groups CTAs.
template <typename T, int NBW>
__global__ void __launch_bounds__(512, 1) k_sweep_cols(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  const int chunk = blockIdx.x % a.P, grp = blockIdx.x / a.P;
  const int r0 = grp * NBW, nb = min(NBW, a.nrhs - r0);
  const int mc = a.mc, mcr = a.mcr;
  const int A = a.ca[chunk], L = a.cb[chunk] - A + 1;
  const int nsteps = 2 * L - 1;
  const int tid = threadIdx.x, nth = blockDim.x;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tv = reinterpret_cast<C*>(smraw);   // [mc][NBW]: T_j
  C* yb = tv + (size_t)mc * NBW;         // [2][mc][NBW]: the blocks of the last two steps
  auto block_of = [&](int q) { return q < L ? A + q : A + (2 * L - 2 - q); };
  ptx::grid_dep_wait();
  ptx::grid_dep_launch();
  for (int q = 0; q < nsteps; ++q) {
    const bool fwd = q < L;
    const int j = block_of(q);
    const C* prev = yb + (size_t)((q - 1) & 1) * mc * NBW;
    C* cur = yb + (size_t)(q & 1) * mc * NBW;
    const size_t oc = (size_t)(fwd ? j - 1 : j) * mc;
    for (int i = tid; i < mc * NBW; i += nth) {
      const int k = i / NBW, r = i - k * NBW;
      C v;
      v.x = 0;
      v.y = 0;
      if (!fwd || q > 0) {
        cmac(v, a.cd[oc + k], prev[i]);
        if (fwd) {  // C_{j-1}^T
          if (k > 0) cmac(v, a.cu[oc + k - 1], prev[i - NBW]);
          if (k + 1 < mc) cmac(v, a.cl[oc + k + 1], prev[i + NBW]);
        } else {    // C_j
          if (k > 0) cmac(v, a.cl[oc + k], prev[i - NBW]);
          if (k + 1 < mc) cmac(v, a.cu[oc + k], prev[i + NBW]);
        }
      }
      if (fwd) {  // a ragged group repeats its last right-hand side
        C t = a.b[(size_t)(r0 + min(r, nb - 1)) * a.Nc + (size_t)j * mc + k];
        t.x -= v.x;
        t.y -= v.y;
        tv[i] = t;
      } else {
        tv[i] = v;
      }
    }
    __syncthreads();
    const C* g = a.Gt + (size_t)j * mc * mcr;
    for (int rr = tid; rr < mc; rr += nth) {
      C acc[NBW];
#pragma unroll
      for (int r = 0; r < NBW; ++r) {
        acc[r].x = 0;
        acc[r].y = 0;
      }
      // blocks of 8 columns; the next block's entries are loaded before the
      // current block's products, so the L2 latency overlaps them
      const int c8 = mc & ~7;
      C gv[8], gn[8];
      if (c8 > 0) {
#pragma unroll
        for (int u = 0; u < 8; ++u) gv[u] = g[(size_t)u * mcr + rr];
      }
      for (int c = 0; c < c8; c += 8) {
        if (c + 8 < c8) {
#pragma unroll
          for (int u = 0; u < 8; ++u) gn[u] = g[(size_t)(c + 8 + u) * mcr + rr];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const C* tc = tv + (size_t)(c + u) * NBW;
#pragma unroll
          for (int r = 0; r < NBW; ++r) cmac(acc[r], gv[u], tc[r]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) gv[u] = gn[u];
      }
      for (int c = c8; c < mc; ++c) {
        const C gc = g[(size_t)c * mcr + rr];
        const C* tc = tv + (size_t)c * NBW;
#pragma unroll
        for (int r = 0; r < NBW; ++r) cmac(acc[r], gc, tc[r]);
      }
#pragma unroll
      for (int r = 0; r < NBW; ++r) {
        C* xo = a.x + (size_t)(r0 + r) * a.Nc + (size_t)j * mc + rr;
        C val = acc[r];
        if (!fwd) {
          C z;
          z.x = 0;
          z.y = 0;
          if (r < nb) z = *xo;  // the padded columns of a ragged group are never stored
          val.x = z.x - acc[r].x;
          val.y = z.y - acc[r].y;
        }
        cur[(size_t)rr * NBW + r] = val;
        if (r < nb) *xo = val;  // z_j forward, y_j backward (y_{A+L-1} = z_{A+L-1})
      }
    }
    __syncthreads();
  }
}

// The separator values xhat = Sinv rhat for a group of NBW right-hand sides per
// CTA and a block of 256 separator unknowns.  The reduced system is the Schur
// complement of the complex-symmetric A_q on the separator rows, so Sinv is
// complex symmetric and its column rr is its row rr: a thread owns unknown rr
// and reads Sinv[c][rr] over c (consecutive across lanes), with the group's
// rhat[c][0..NBW-1] staged in shared memory in slices of 1024 columns.
template <typename T, int NBW>
__global__ void __launch_bounds__(256) k_sep_cols(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  constexpr int KS = 1024;
  ptx::grid_dep_wait();  // launched with a programmatic dependency inside the cycle
  ptx::grid_dep_launch();
  const int groups = (a.nrhs + NBW - 1) / NBW;
  const int blk = blockIdx.x / groups, grp = blockIdx.x - blk * groups;
  const int r0 = grp * NBW, nb = min(NBW, a.nrhs - r0);
  const int tid = threadIdx.x, nth = blockDim.x;
  const int rr = blk * 256 + tid;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* hs = reinterpret_cast<C*>(smraw);  // [KS][NBW]
  C acc[NBW];
#pragma unroll
  for (int r = 0; r < NBW; ++r) {
    acc[r].x = 0;
    acc[r].y = 0;
  }
  for (int k0 = 0; k0 < a.nred; k0 += KS) {
    const int kn = min(KS, a.nred - k0);
    __syncthreads();
    for (int i = tid; i < kn * NBW; i += nth) {
      const int c = i / NBW, r = i - c * NBW;
      C v;
      v.x = 0;
      v.y = 0;
      if (r < nb) v = a.rhat[(size_t)(r0 + r) * a.nred + k0 + c];
      hs[i] = v;
    }
    __syncthreads();
    if (rr < a.nred) {
      const C* sc = a.Sinv + (size_t)k0 * a.ldS + rr;
      const int c8 = kn & ~7;
      C sv[8], sn[8];
      if (c8 > 0) {
#pragma unroll
        for (int u = 0; u < 8; ++u) sv[u] = sc[(size_t)u * a.ldS];
      }
      for (int c = 0; c < c8; c += 8) {
        if (c + 8 < c8) {  // the next block's entries ahead of this block's products
#pragma unroll
          for (int u = 0; u < 8; ++u) sn[u] = sc[(size_t)(c + 8 + u) * a.ldS];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const C* hc = hs + (size_t)(c + u) * NBW;
#pragma unroll
          for (int r = 0; r < NBW; ++r) cmac(acc[r], sv[u], hc[r]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) sv[u] = sn[u];
      }
      for (int c = c8; c < kn; ++c) {
        const C sv = sc[(size_t)c * a.ldS];
        const C* hc = hs + (size_t)c * NBW;
#pragma unroll
        for (int r = 0; r < NBW; ++r) cmac(acc[r], sv, hc[r]);
      }
    }
  }
  if (rr < a.nred) {
    const int k = rr / a.mc, e = rr - k * a.mc;
#pragma unroll
    for (int r = 0; r < NBW; ++r)
      if (r < nb) a.x[(size_t)(r0 + r) * a.Nc + (size_t)a.sep[k] * a.mc + e] = acc[r];
  }
}

// The spike correction x_j -= [L_j | R_j] [x_left; x_right] for a group of NBW
// right-hand sides per CTA, from the spikes stored transposed (LRt[j][col][row],
// rows padded to mcr): one CTA per (chunk row j, group), the groups of one j
// adjacent in the grid so that they read LRt[j] together through L2; a thread
// owns a row and NBW accumulators and reads its row's entries (consecutive
// across lanes) and the separator values of its group from shared memory.
template <typename T, int NBW>
__global__ void __launch_bounds__(512) k_spikes_cols(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  ptx::grid_dep_wait();  // launched with a programmatic dependency inside the cycle
  ptx::grid_dep_launch();
  const int groups = (a.nrhs + NBW - 1) / NBW;
  const int j = blockIdx.x / groups, grp = blockIdx.x - j * groups;
  const int chunk = a.chunk_of[j];
  if (chunk < 0) return;  // a separator row (uniform over the CTA)
  const int r0 = grp * NBW, nb = min(NBW, a.nrhs - r0);
  const int mc = a.mc, mcp = a.mcp, K = 2 * mcp;
  const int tid = threadIdx.x, nth = blockDim.x;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* xs = reinterpret_cast<C*>(smraw);  // [K][NBW]
  for (int i = tid; i < K * NBW; i += nth) {
    const int col = i / NBW, r = i - col * NBW;
    const int side = col >= mcp ? 1 : 0, k = col - side * mcp;
    const bool has = r < nb && k < mc && (side == 0 ? chunk > 0 : chunk < a.P - 1);
    C v;
    v.x = 0;
    v.y = 0;
    if (has) v = a.x[(size_t)(r0 + r) * a.Nc + (size_t)a.sep[side == 0 ? chunk - 1 : chunk] * mc + k];
    xs[i] = v;
  }
  __syncthreads();
  const C* lr = a.LRt + (size_t)j * K * a.mcr;
  for (int rr = tid; rr < mc; rr += nth) {
    C acc[NBW];
#pragma unroll
    for (int r = 0; r < NBW; ++r) {
      acc[r].x = 0;
      acc[r].y = 0;
    }
    const int c8 = K & ~7;
    C lv[8], ln[8];
    if (c8 > 0) {
#pragma unroll
      for (int u = 0; u < 8; ++u) lv[u] = lr[(size_t)u * a.mcr + rr];
    }
    for (int c = 0; c < c8; c += 8) {
      if (c + 8 < c8) {  // the next block's entries ahead of this block's products
#pragma unroll
        for (int u = 0; u < 8; ++u) ln[u] = lr[(size_t)(c + 8 + u) * a.mcr + rr];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const C* xc = xs + (size_t)(c + u) * NBW;
#pragma unroll
        for (int r = 0; r < NBW; ++r) cmac(acc[r], lv[u], xc[r]);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) lv[u] = ln[u];
    }
    for (int c = c8; c < K; ++c) {
      const C lc = lr[(size_t)c * a.mcr + rr];
      const C* xc = xs + (size_t)c * NBW;
#pragma unroll
      for (int r = 0; r < NBW; ++r) cmac(acc[r], lc, xc[r]);
    }
#pragma unroll
    for (int r = 0; r < NBW; ++r) {
      if (r < nb) {
        C* xo = a.x + (size_t)(r0 + r) * a.Nc + (size_t)j * mc + rr;
        C v = *xo;
        v.x -= acc[r].x;
        v.y -= acc[r].y;
        *xo = v;
      }
    }
  }
}

// Tall-skinny products of the reduced solve and of the spike correction, for
// one right-hand side or a tile of NB:
//   MODE 0: xhat = Sinv rhat, written into the separator rows of x (one CTA per
//           16 rows of Sinv, whose rows are padded to an even length ldS);
//   MODE 1: x_j -= [L_j | R_j] [x_left; x_right] on every chunk row j (one CTA
//           per 32 rows (one rhs: 16 warps of two rows, a single pass) or per
//           half (tiles) of a block row; a CTA of a separator row returns at once).
// The CTA stages the tile's right-hand-side columns in shared memory ([rhs]
// [column]); each warp streams R matrix rows two complex values per lane and
// load (16-byte loads for FP32, consecutive across lanes), reads the matching
// column pair of every right-hand side with one shared load, and keeps R x NB
// accumulators; row sums are warp reductions in a fixed order.  The tile index
// varies fastest in the grid, so concurrent CTAs of different tiles read the
// same matrix rows through L2.
__device__ __forceinline__ void ld_pair(const float2* p, float2& u, float2& v) {
  const float4 w = *reinterpret_cast<const float4*>(p);
  u = make_float2(w.x, w.y);
  v = make_float2(w.z, w.w);
}
__device__ __forceinline__ void ld_pair(const double2* p, double2& u, double2& v) {
  u = p[0];
  v = p[1];
}

template <typename T, int NB, int MODE>
__global__ void __launch_bounds__(512) k_coarse_tsgemm(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  ptx::grid_dep_wait();  // launched with a programmatic dependency inside the cycle
  ptx::grid_dep_launch();
  constexpr int R = MODE == 0 ? 1 : 2, WARPS = 16;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* Xs = reinterpret_cast<C*>(smraw);  // [NB][kc]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ntiles = (a.nrhs + NB - 1) / NB;
  const int tile = blockIdx.x % ntiles, blk = blockIdx.x / ntiles;
  const int r0 = tile * NB, nb = min(NB, a.nrhs - r0);
  const int mc = a.mc, mcp = a.mcp;
  int K, kc, rbeg, rend, j = 0, chunk = 0;
  if (MODE == 0) {
    K = a.ldS;
    kc = NB == 1 ? K : 1024;
    rbeg = blk * WARPS * R;
    rend = min(a.nred, rbeg + WARPS * R);
  } else {
    // CTAs per block row: one right-hand side, 32 rows each (16 warps of two rows, one pass)
    const int PARTS = NB == 1 ? (mc + 31) / 32 : 2;
    j = blk / PARTS;
    chunk = a.chunk_of[j];
    if (chunk < 0) return;  // separator block row (uniform over the CTA)
    const int hr = (mc + PARTS - 1) / PARTS;
    K = 2 * mcp;
    kc = K;
    rbeg = (blk - j * PARTS) * hr;
    rend = min(mc, rbeg + hr);
  }
  auto stage = [&](int k0, int kn) {
    for (int i = tid; i < NB * kn; i += blockDim.x) {
      const int r = i / kn, c = i - r * kn;
      C v;
      v.x = 0;
      v.y = 0;
      if (r < nb) {
        if (MODE == 0) {
          if (k0 + c < a.nred) v = a.rhat[(size_t)(r0 + r) * a.nred + k0 + c];
        } else {
          const int side = c >= mcp ? 1 : 0, k = c - side * mcp;
          const bool has = k < mc && (side == 0 ? chunk > 0 : chunk < a.P - 1);
          if (has) v = a.x[(size_t)(r0 + r) * a.Nc + (size_t)a.sep[side == 0 ? chunk - 1 : chunk] * mc + k];
        }
      }
      Xs[(size_t)r * kc + c] = v;
    }
  };
  auto rowptr = [&](int row) -> const C* {
    return MODE == 0 ? a.Sinv + (size_t)row * a.ldS : a.LR + ((size_t)j * mc + row) * 2 * mcp;
  };
  // acc[q][r] += sum over the column pairs [k0, k0 + kn) of A[row_q] X_r
  auto dot = [&](C (&acc)[R][NB], const C* const (&rows)[R], int k0, int kn) {
#pragma unroll(NB == 1 ? 4 : 2)
    for (int c = 2 * lane; c < kn; c += 64) {
      C u[R], v[R];
#pragma unroll
      for (int q = 0; q < R; ++q) ld_pair(rows[q] + k0 + c, u[q], v[q]);
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        C xu, xv;
        ld_pair(Xs + (size_t)r * kc + c, xu, xv);
#pragma unroll
        for (int q = 0; q < R; ++q) {
          cmac(acc[q][r], u[q], xu);
          cmac(acc[q][r], v[q], xv);
        }
      }
    }
  };
  // lane r < nb ends with the sums of right-hand side r; MODE 1 subtracts them
  // from y values the lane loaded before the products (yv), so no load waits
  // behind a store
  auto finish = [&](C (&acc)[R][NB], int row_first, const C (&yv)[R]) {
    C out[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      out[q].x = 0;
      out[q].y = 0;
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        const C s = warp_sum<T>(acc[q][r]);
        if (lane == r) out[q] = s;
      }
    }
    if (lane >= nb) return;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int row = row_first + q;
      if (row >= rend) continue;
      if (MODE == 0) {
        const int k = row / mc, e = row - k * mc;
        a.x[(size_t)(r0 + lane) * a.Nc + (size_t)a.sep[k] * mc + e] = out[q];
      } else {
        C v = yv[q];
        v.x -= out[q].x;
        v.y -= out[q].y;
        a.x[(size_t)(r0 + lane) * a.Nc + (size_t)j * mc + row] = v;
      }
    }
  };
  auto zero = [&](C (&acc)[R][NB]) {
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        acc[q][r].x = 0;
        acc[q][r].y = 0;
      }
  };
  C acc[R][NB];
  if (MODE == 0) {
    const int row = rbeg + warp;
    const C* rows[R] = {rowptr(row < rend ? row : rbeg)};
    const C none[R] = {};
    zero(acc);
    for (int k0 = 0; k0 < K; k0 += kc) {
      const int kn = min(kc, K - k0);
      __syncthreads();
      stage(k0, kn);
      __syncthreads();
      dot(acc, rows, k0, kn);
    }
    finish(acc, row, none);
  } else {
    stage(0, K);
    __syncthreads();
    for (int e0 = rbeg + warp * R; e0 < rend; e0 += WARPS * R) {
      const C* rows[R];
      C yv[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        rows[q] = rowptr(e0 + q < rend ? e0 + q : e0);
        yv[q].x = 0;
        yv[q].y = 0;
        if (lane < nb && e0 + q < rend) yv[q] = a.x[(size_t)(r0 + lane) * a.Nc + (size_t)j * mc + e0 + q];
      }
      zero(acc);
      dot(acc, rows, 0, K);
      finish(acc, e0, yv);
    }
  }
}

// separator product on tiles of NB0 right-hand sides, spike correction on tiles of NB1
template <typename T, int NB0, int NB1 = NB0>
static cudaError_t launch_tsgemm(const CoarsePartArgs<T>& a, cudaStream_t s) {
  using C = typename Cx<T>::t;
  const int nt0 = (a.nrhs + NB0 - 1) / NB0, nt1 = (a.nrhs + NB1 - 1) / NB1;
  const size_t sm0 = sizeof(C) * (size_t)NB0 * (NB0 == 1 ? a.ldS : 1024), sm1 = sizeof(C) * (size_t)NB1 * 2 * a.mcp;
  cudaError_t e = cudaFuncSetAttribute(k_coarse_tsgemm<T, NB0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm0);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_coarse_tsgemm<T, NB1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
  if (e != cudaSuccess) return e;
  const unsigned g0 = (unsigned)((a.nred + 15) / 16) * nt0;
  e = launch_pdl(k_coarse_tsgemm<T, NB0, 0>, dim3(g0), dim3(512), sm0, s, 0, a);
  if (e != cudaSuccess) return e;
  const unsigned g1 = (unsigned)((NB1 == 1 ? (a.mc + 31) / 32 : 2) * a.mc) * nt1;
  return launch_pdl(k_coarse_tsgemm<T, NB1, 1>, dim3(g1), dim3(512), sm1, s, 0, a);
}

// The separator values xhat = Sinv rhat for one right-hand side from the upper
// triangle of Sinv only.  Sinv is complex symmetric (Sinv^T = Sinv: the inverse
// of the Schur complement of the complex-symmetric A_q), so a stored block
// S_IJ (J > I) of 64 x 64 serves both y_I += S_IJ x_J and y_J += S_IJ^T x_I:
// half the bytes of the full GEMV.  One CTA per stored block stages it in
// shared memory (rows padded to 65 entries, so that neither the row-wise nor
// the column-wise pass has more than the minimum two wavefronts per warp),
// forms both products and writes them as partials part[(I T + J) 64 + r] (for
// row tile I); k_sep_sym_sum adds the T partials of every unknown in a fixed
// order and writes it into the separator rows of x.
template <typename T>
__global__ void __launch_bounds__(256) k_sep_sym(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  constexpr int R = 64, RS = 65;
  __shared__ C sb[R * RS];
  __shared__ C xi[R], xj[R];
  __shared__ C red[4][R];
  ptx::grid_dep_wait();  // launched with a programmatic dependency inside the cycle
  ptx::grid_dep_launch();
  const int2 ij = a.sym_ij[blockIdx.x];
  const int I = ij.x, J = ij.y, tid = threadIdx.x;
  const C* blk = a.Ssym + (size_t)blockIdx.x * R * R;
  for (int e = tid; e < R * R / 2; e += 256) {  // two complex values per 16-byte load
    const int r = e / (R / 2), c2 = e - r * (R / 2);
    const C* p = blk + (size_t)r * R + 2 * c2;
    sb[r * RS + 2 * c2] = p[0];
    sb[r * RS + 2 * c2 + 1] = p[1];
  }
  if (tid < R) {
    C v;
    v.x = 0;
    v.y = 0;
    const int gi = I * R + tid, gj = J * R + tid;
    xi[tid] = gi < a.nred ? a.rhat[gi] : v;
    xj[tid] = gj < a.nred ? a.rhat[gj] : v;
  }
  __syncthreads();
  const int r = tid & (R - 1), q = tid >> 6;  // row (or column) and quarter of the 64
  C acc;
  acc.x = 0;
  acc.y = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) cmac(acc, sb[r * RS + q * 16 + k], xj[q * 16 + k]);  // (S_IJ x_J)_r
  red[q][r] = acc;
  __syncthreads();
  if (tid < R) {
    C y = red[0][tid];
#pragma unroll
    for (int u = 1; u < 4; ++u) {
      y.x += red[u][tid].x;
      y.y += red[u][tid].y;
    }
    a.spart[((size_t)I * a.Tsym + J) * R + tid] = y;
  }
  if (J == I) return;  // uniform over the CTA
  __syncthreads();
  acc.x = 0;
  acc.y = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) cmac(acc, sb[(q * 16 + k) * RS + r], xi[q * 16 + k]);  // (S_IJ^T x_I)_c, c = r
  red[q][r] = acc;
  __syncthreads();
  if (tid < R) {
    C y = red[0][tid];
#pragma unroll
    for (int u = 1; u < 4; ++u) {
      y.x += red[u][tid].x;
      y.y += red[u][tid].y;
    }
    a.spart[((size_t)J * a.Tsym + I) * R + tid] = y;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sep_sym_sum(const CoarsePartArgs<T> a) {
  using C = typename Cx<T>::t;
  ptx::grid_dep_wait();
  ptx::grid_dep_launch();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.nred) return;
  const int I = idx >> 6, r = idx & 63;
  C y;
  y.x = 0;
  y.y = 0;
  for (int J = 0; J < a.Tsym; ++J) {
    const C v = a.spart[((size_t)I * a.Tsym + J) * 64 + r];
    y.x += v.x;
    y.y += v.y;
  }
  const int k = idx / a.mc, e = idx - k * a.mc;
  a.x[(size_t)a.sep[k] * a.mc + e] = y;
}

// ------------------------------------------------------------- launcher
template <typename T>
size_t chunk_sweep2_smem(const CoarsePartArgs<T>& a) {
  using C = typename Cx<T>::t;
  return 16 + sizeof(C) * ((size_t)3 * a.rpc * a.mcp + (size_t)11 * a.mc + (size_t)a.Lmax * a.rpc);
}

template <typename T>
size_t chunk_sweep_smem(const CoarsePartArgs<T>& a, bool prefetch) {
  using C = typename Cx<T>::t;
  size_t s = sizeof(C) * ((size_t)11 * a.mc + (size_t)a.Lmax * a.rpc);
  if (prefetch) s += sizeof(C) * (size_t)2 * a.rpc * a.mcp;
  return s;
}

template <typename K, typename Args>
static cudaError_t launch_cluster(K kern, const Args& a, int grid, int cluster, size_t smem, cudaStream_t s,
                                  int threads = 512) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
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
constexpr int mr_tile() { return sizeof(T) == 8 ? 4 : 8; }

template <typename T, int NB>
size_t chunk_sweep_mr_smem(const CoarsePartArgs<T>& a, bool prefetch) {
  using C = typename Cx<T>::t;
  size_t s = (size_t)2 * a.mc * NB + (size_t)6 * a.mc + (size_t)2 * a.mc * NB + (size_t)a.mc * NB +
             (size_t)16 * a.rpcm * (NB + 1) + (size_t)a.Lmax * a.rpcm * NB;
  if (prefetch) s += (size_t)2 * a.mc * a.rpcm;
  return s * sizeof(C);
}

// many right-hand sides: tiles of NB per cluster / warp
template <typename T, int NB>
static cudaError_t launch_coarse_part_mr_nb(const CoarsePartArgs<T>& a, int cluster, cudaStream_t s) {
  const int ntiles = (a.nrhs + NB - 1) / NB;
  const bool pf = chunk_sweep_mr_smem<T, NB>(a, true) <= 220 * 1024;
  const size_t sm1 = chunk_sweep_mr_smem<T, NB>(a, pf);
  if (sm1 > 227 * 1024) return cudaErrorInvalidValue;
  const int grid = cluster * a.P * ntiles;
  cudaError_t e = pf ? launch_cluster(k_chunk_sweep_mr<T, NB, true>, a, grid, cluster, sm1, s)
                     : launch_cluster(k_chunk_sweep_mr<T, NB, false>, a, grid, cluster, sm1, s);
  if (e != cudaSuccess || a.P < 2) return e;
  dim3 g1((unsigned)((a.nred + 255) / 256), a.nrhs);
  k_reduced_rhs<T><<<g1, 256, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_tsgemm<T, NB>(a, s);
}

// the widest tile whose sweep buffers fit shared memory (large coarse grids,
// e.g. 401 rows per block, take narrower tiles)
template <typename T>
static cudaError_t launch_coarse_part_mr(const CoarsePartArgs<T>& a, int cluster, cudaStream_t s) {
  constexpr int NB = mr_tile<T>();
  if (chunk_sweep_mr_smem<T, NB>(a, false) <= 227 * 1024) return launch_coarse_part_mr_nb<T, NB>(a, cluster, s);
  if (chunk_sweep_mr_smem<T, NB / 2>(a, false) <= 227 * 1024) return launch_coarse_part_mr_nb<T, NB / 2>(a, cluster, s);
  if (chunk_sweep_mr_smem<T, NB / 4>(a, false) <= 227 * 1024) return launch_coarse_part_mr_nb<T, NB / 4>(a, cluster, s);
  return cudaErrorInvalidValue;
}

// many right-hand sides in groups of NBW per CTA (one CTA per chunk and group),
// then the reduced system and the spike correction on tiles of right-hand sides
template <typename T, int NBW>
static cudaError_t launch_coarse_part_cols(const CoarsePartArgs<T>& a, cudaStream_t s) {
  using C = typename Cx<T>::t;
  const size_t smem = sizeof(C) * (size_t)3 * a.mc * NBW;
  if (smem > 227 * 1024 || a.mc > 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_sweep_cols<T, NBW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int groups = (a.nrhs + NBW - 1) / NBW;
  e = launch_pdl(k_sweep_cols<T, NBW>, dim3(a.P * groups), dim3(512), smem, s, 0, a);
  if (e != cudaSuccess || a.P < 2) return e;
  dim3 g1((unsigned)((a.nred + 255) / 256), a.nrhs);
  if constexpr (std::is_same<T, float>::value) {
    if (a.multi_variant == 2 && a.umma && a.rst) {
      // the separator product and the spike correction on the tensor cores
      // (BF16 reduced inverse and spikes, coarse_umma.cu)
      e = launch_pdl(k_reduced_rhs<T>, g1, dim3(256), 0, s, 0, a);
      if (e != cudaSuccess) return e;
      CoarseUmmaArgs u = *a.umma;
      u.x = a.x;
      u.nrhs = a.nrhs;
      u.err = a.err;
      const int sms = a.nsm > 0 ? a.nsm : 152;
      e = launch_coarse_umma(u, 0, sms, s);
      if (e != cudaSuccess) return e;
      return launch_coarse_umma(u, 1, sms, s);
    }
  }
  {
    CoarsePartArgs<T> b = a;
    b.rst = nullptr;
    e = launch_pdl(k_reduced_rhs<T>, g1, dim3(256), 0, s, 0, b);
  }
  if (e != cudaSuccess) return e;
  // the spike correction in the same groups from the transposed spikes when the
  // context keeps them; else the tiled products (below)
  if (a.LRt) {
    using C = typename Cx<T>::t;
    const int groups = (a.nrhs + NBW - 1) / NBW;
    const size_t sm0 = sizeof(C) * (size_t)1024 * NBW, sm1 = sizeof(C) * (size_t)2 * a.mcp * NBW;
    if (sm1 <= 220 * 1024) {
      e = cudaFuncSetAttribute(k_sep_cols<T, NBW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm0);
      if (e != cudaSuccess) return e;
      e = launch_pdl(k_sep_cols<T, NBW>, dim3((unsigned)((a.nred + 255) / 256 * groups)), dim3(256), sm0, s, 0, a);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(k_spikes_cols<T, NBW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
      if (e != cudaSuccess) return e;
      return launch_pdl(k_spikes_cols<T, NBW>, dim3((unsigned)(a.mc * groups)), dim3(512), sm1, s, 0, a);
    }
  }
  return launch_tsgemm<T, mr_tile<T>()>(a, s);
}

template <typename T>
cudaError_t launch_coarse_part(const CoarsePartArgs<T>& a0, int nrhs, int cluster, cudaStream_t s) {
  // the BF16 staging of the reduced right-hand sides serves the tensor-core path only
  CoarsePartArgs<T> a = a0;
  const bool tc = a.multi_variant == 2 && nrhs >= 8 && a.umma && a.rst;
  if (!tc) a.rst = nullptr;
  if (nrhs >= 2 && a.Gt) {
    CoarsePartArgs<T> b = a;
    b.nrhs = nrhs;
    if (a.multi_variant >= 1 && nrhs >= 8) {
      // the narrowest group width with at most one CTA per SM: P * ceil(nrhs / NBW) <= SMs
      const int per = std::max(1, (a.nsm > 0 ? a.nsm : 152) / std::max(1, a.P));
      const int need = (nrhs + per - 1) / per;
      cudaError_t e = cudaErrorInvalidValue;
      if (need <= 8) e = launch_coarse_part_cols<T, 8>(b, s);
      else if (need <= 10) e = launch_coarse_part_cols<T, 10>(b, s);
      else if (need <= 12) e = launch_coarse_part_cols<T, 12>(b, s);
      else if (need <= 16) e = launch_coarse_part_cols<T, 16>(b, s);
      if (e != cudaErrorInvalidValue) return e;
    }
    b.rst = nullptr;
    return launch_coarse_part_mr<T>(b, cluster, s);
  }
  const bool pf = chunk_sweep_smem(a, true) <= 220 * 1024;
  const size_t sm1 = chunk_sweep_smem(a, pf);
  cudaError_t e;
  if (a.sweep_variant == 2 && a.mc <= 256 && a.rpc <= 32 && chunk_sweep2_smem(a) <= 220 * 1024 && a.err) {
    cudaError_t e2 = cudaFuncSetAttribute(k_chunk_sweep2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)chunk_sweep2_smem(a));
    if (e2 != cudaSuccess) return e2;
    e = launch_pdl(k_chunk_sweep2<T>, dim3(cluster * a.P * nrhs), dim3(1024), chunk_sweep2_smem(a), s, cluster, a,
                   a.err);
  } else if (a.sweep_variant == 1 && a.mc <= 256 && a.rpc <= 32) {
    e = pf ? launch_cluster(k_chunk_sweep1<T, true>, a, cluster * a.P * nrhs, cluster, sm1, s, 1024)
           : launch_cluster(k_chunk_sweep1<T, false>, a, cluster * a.P * nrhs, cluster, sm1, s, 1024);
  } else {
    e = pf ? launch_cluster(k_chunk_sweep<T, true>, a, cluster * a.P * nrhs, cluster, sm1, s)
           : launch_cluster(k_chunk_sweep<T, false>, a, cluster * a.P * nrhs, cluster, sm1, s);
  }
  if (e != cudaSuccess || a.P < 2) return e;
  dim3 g1((unsigned)((a.nred + 255) / 256), nrhs);
  e = launch_pdl(k_reduced_rhs<T>, g1, dim3(256), 0, s, 0, a);
  if (e != cudaSuccess) return e;
  CoarsePartArgs<T> b = a;
  b.nrhs = nrhs;
  if constexpr (std::is_same<T, float>::value) {
    if (nrhs == 1 && a.Ssym && a.spart && a.sym_ij) {
      // the separator values from Sinv's upper triangle, then the spike correction
      e = launch_pdl(k_sep_sym<T>, dim3((unsigned)a.nsym), dim3(256), 0, s, 0, b);
      if (e != cudaSuccess) return e;
      e = launch_pdl(k_sep_sym_sum<T>, dim3((unsigned)((a.nred + 255) / 256)), dim3(256), 0, s, 0, b);
      if (e != cudaSuccess) return e;
      using C = typename Cx<T>::t;
      const size_t sm1 = sizeof(C) * (size_t)2 * a.mcp;
      e = cudaFuncSetAttribute(k_coarse_tsgemm<T, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
      if (e != cudaSuccess) return e;
      return launch_pdl(k_coarse_tsgemm<T, 1, 1>, dim3((unsigned)((a.mc + 31) / 32 * a.mc)), dim3(512), sm1, s, 0,
                        b);
    }
  }
  return launch_tsgemm<T, 1>(b, s);
}

template cudaError_t launch_coarse_part<double>(const CoarsePartArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_coarse_part<float>(const CoarsePartArgs<float>&, int, int, cudaStream_t);

}  // namespace th
