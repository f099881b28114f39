// K3/K4: the complex-shifted domain-decomposition smoother (Section 4.1,
// Algorithm 2, Eq. RAS_like_update) applied with precomputed inverse rows.
//
// With v = 0 on entry (the first DDStep of a CSDDSmoother), the local solve
// of subdomain i reduces to w_i = (A_s^(i))^{-1} R_i r, and only its values on
// Dofs(U^(i)) are ever used.  The set-up stores exactly those rows, scaled by
// 1/L_j, as W_i (NR x NC, NR = Lu^2 U-box nodes, NC = Lw^2 Omega-box nodes).
//
// K3 (k_dd_apply): per subdomain, gather x = R_i r (the Omega box of r, L2
// resident) into shared memory and stream W_i from HBM: V_i = W_i x.  W_i is
// stored chunk-major, [chunk][row] of 16-byte chunks holding CPC consecutive
// columns of one row (CPC = 1 complex FP64, 2 FP32, 4 BF16/FP16), so a warp
// reads 512 contiguous bytes per load.  Thread (row, g) accumulates the
// chunks g, g + G, ... of its row; the G partial sums are added in a fixed
// order.  Low-precision rows are widened to FP32 and accumulated in FP32.
//
// K4 (k_dd_combine): u_j (+)= sum over the (at most four) subdomains whose
// U box holds j of V_i[j], in a fixed order (bitwise deterministic).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "kernels.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace th {

template <int KIND> struct WTraits;
template <> struct WTraits<W_FP64> { static constexpr int CPC = 1; };
template <> struct WTraits<W_FP32> { static constexpr int CPC = 2; };
template <> struct WTraits<W_BF16> { static constexpr int CPC = 4; };
template <> struct WTraits<W_FP16> { static constexpr int CPC = 4; };

template <typename T, int KIND>
__device__ __forceinline__ void unpack_chunk(const void* base, size_t idx, T* wr, T* wi) {
  if constexpr (KIND == W_FP64) {
    const double2 v = __ldcs(reinterpret_cast<const double2*>(base) + idx);
    wr[0] = (T)v.x;
    wi[0] = (T)v.y;
  } else if constexpr (KIND == W_FP32) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(base) + idx);
    wr[0] = v.x; wi[0] = v.y; wr[1] = v.z; wi[1] = v.w;
  } else if constexpr (KIND == W_BF16) {
    const uint4 v = __ldcs(reinterpret_cast<const uint4*>(base) + idx);
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      wr[j] = __uint_as_float(w[j] << 16);
      wi[j] = __uint_as_float(w[j] & 0xffff0000u);
    }
  } else {
    const uint4 v = __ldcs(reinterpret_cast<const uint4*>(base) + idx);
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __half2 h2 = *reinterpret_cast<const __half2*>(&w[j]);
      float2 f = __half22float2(h2);
      wr[j] = f.x;
      wi[j] = f.y;
    }
  }
}

// same unpacking from shared memory (plain loads)
template <typename T, int KIND>
__device__ __forceinline__ void unpack_chunk_smem(const void* base, size_t idx, T* wr, T* wi) {
  if constexpr (KIND == W_FP64) {
    const double2 v = reinterpret_cast<const double2*>(base)[idx];
    wr[0] = (T)v.x;
    wi[0] = (T)v.y;
  } else if constexpr (KIND == W_FP32) {
    const float4 v = reinterpret_cast<const float4*>(base)[idx];
    wr[0] = v.x; wi[0] = v.y; wr[1] = v.z; wi[1] = v.w;
  } else if constexpr (KIND == W_BF16) {
    const uint4 v = reinterpret_cast<const uint4*>(base)[idx];
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      wr[j] = __uint_as_float(w[j] << 16);
      wi[j] = __uint_as_float(w[j] & 0xffff0000u);
    }
  } else {
    const uint4 v = reinterpret_cast<const uint4*>(base)[idx];
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __half2 h2 = *reinterpret_cast<const __half2*>(&w[j]);
      float2 f = __half22float2(h2);
      wr[j] = f.x;
      wi[j] = f.y;
    }
  }
}

template <typename T, int KIND, int NRHS, int MAXT>
__global__ void __launch_bounds__(MAXT) k_dd_apply(const DDArgs<T> a) {
  using C = typename Cx<T>::t;
  constexpr int CPC = WTraits<KIND>::CPC;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int XL = a.NCH * CPC;
  C* xs = reinterpret_cast<C*>(smraw);        // [NRHS][XL]
  C* red = xs + NRHS * XL;                     // [G][NR][NRHS]
  const int tid = threadIdx.x, nth = blockDim.x;
  const int rr = tid % a.NR, g = tid / a.NR;
  const int r0 = blockIdx.y * NRHS;
  const int nr = min(NRHS, a.nrhs - r0);
  ptx::grid_dep_wait();  // launched with a programmatic dependency inside the cycle
  ptx::grid_dep_launch();
  for (int sub = blockIdx.x; sub < a.nsub; sub += gridDim.x) {
    const int* bb = a.box + (size_t)sub * 12;
    const int ox = bb[0], oy = bb[1], wx = bb[2], wy = bb[3], oz = bb[8], wz = bb[9];
    const int L2 = a.Lw * a.Lw;
    for (int i = tid; i < NRHS * XL; i += nth) {
      const int k = i / XL, c = i - k * XL;
      const int cz = c / L2, cr = c - cz * L2;
      const int cy = cr / a.Lw, cx = cr - cy * a.Lw;
      C v;
      v.x = 0;
      v.y = 0;
      if (k < nr && c < a.NC && cx < wx && cy < wy && cz < wz)
        v = a.r[(size_t)(r0 + k) * a.N + ((size_t)(oz + cz) * a.m + (oy + cy)) * a.m + (ox + cx)];
      xs[i] = v;
    }
    __syncthreads();
    if (g < a.G) {
      T acr[NRHS], aci[NRHS];
#pragma unroll
      for (int k = 0; k < NRHS; ++k) { acr[k] = 0; aci[k] = 0; }
      const size_t wbase = (size_t)sub * a.NCH * a.NR + rr;
#pragma unroll 4
      for (int ch = g; ch < a.NCH; ch += a.G) {
        T wr[CPC], wi[CPC];
        unpack_chunk<T, KIND>(a.W, wbase + (size_t)ch * a.NR, wr, wi);
#pragma unroll
        for (int j = 0; j < CPC; ++j) {
#pragma unroll
          for (int k = 0; k < NRHS; ++k) {
            const C xv = xs[k * XL + ch * CPC + j];
            acr[k] = fmadd(wr[j], xv.x, acr[k]);
            acr[k] = fmadd(-wi[j], xv.y, acr[k]);
            aci[k] = fmadd(wr[j], xv.y, aci[k]);
            aci[k] = fmadd(wi[j], xv.x, aci[k]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < NRHS; ++k) {
        C v;
        v.x = acr[k];
        v.y = aci[k];
        red[((size_t)g * a.NR + rr) * NRHS + k] = v;
      }
    }
    __syncthreads();
    if (tid < a.NR) {
      const T sc = a.wscale ? (T)a.wscale[sub] : (T)1;
      for (int k = 0; k < nr; ++k) {
        T sr = 0, si = 0;
        for (int gg = 0; gg < a.G; ++gg) {
          const C v = red[((size_t)gg * a.NR + tid) * NRHS + k];
          sr += v.x;
          si += v.y;
        }
        C o;
        o.x = sr * sc;
        o.y = si * sc;
        a.V[((size_t)(r0 + k) * a.nsub + sub) * a.NR + tid] = o;
      }
    }
    __syncthreads();
  }
}

template <typename T, int KIND, int NRHS, int MAXT>
static cudaError_t launch_dd_kt(const DDArgs<T>& a, int grid_cap, int threads, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_dd_apply<T, KIND, NRHS, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int gx = (grid_cap > 0 && grid_cap < a.nsub) ? grid_cap : a.nsub;
  dim3 grid(gx, (a.nrhs + NRHS - 1) / NRHS);
  return launch_pdl(k_dd_apply<T, KIND, NRHS, MAXT>, grid, dim3(threads), smem, s, 0, a);
}

// up to 512 threads (U boxes of at most 512 nodes, G column groups), or 1024
// threads with one column group for larger boxes (e.g. 6 cells of order 6)
template <typename T, int KIND, int NRHS>
static cudaError_t launch_dd_k(const DDArgs<T>& a, int grid_cap, cudaStream_t s) {
  using C = typename Cx<T>::t;
  constexpr int CPC = WTraits<KIND>::CPC;
  const int threads = ((a.NR * a.G + 31) / 32) * 32;
  if (threads > 1024) return cudaErrorInvalidConfiguration;
  const size_t smem = sizeof(C) * ((size_t)NRHS * a.NCH * CPC + (size_t)a.G * a.NR * NRHS);
  if (threads > 512) return launch_dd_kt<T, KIND, NRHS, 1024>(a, grid_cap, threads, smem, s);
  return launch_dd_kt<T, KIND, NRHS, 512>(a, grid_cap, threads, smem, s);
}

// shared memory of k_dd_apply for NRHS right-hand sides per CTA
template <typename T, int KIND>
static size_t dd_apply_smem(const DDArgs<T>& a, int nrhs) {
  using C = typename Cx<T>::t;
  return sizeof(C) * ((size_t)nrhs * a.NCH * WTraits<KIND>::CPC + (size_t)a.G * a.NR * nrhs);
}

template <typename T, int KIND>
static cudaError_t launch_dd_kind(const DDArgs<T>& a, int grid_cap, cudaStream_t s) {
  if (a.nrhs >= 8 && dd_apply_smem<T, KIND>(a, 8) <= 227 * 1024) return launch_dd_k<T, KIND, 8>(a, grid_cap, s);
  if (a.nrhs >= 4) return launch_dd_k<T, KIND, 4>(a, grid_cap, s);
  if (a.nrhs >= 2) return launch_dd_k<T, KIND, 2>(a, grid_cap, s);
  return launch_dd_k<T, KIND, 1>(a, grid_cap, s);
}

template <>
cudaError_t launch_dd_apply<double>(const DDArgs<double>& a, int kind, int grid_cap, cudaStream_t s) {
  if (kind != W_FP64) return cudaErrorInvalidValue;
  return launch_dd_kind<double, W_FP64>(a, grid_cap, s);
}

template <>
cudaError_t launch_dd_apply<float>(const DDArgs<float>& a, int kind, int grid_cap, cudaStream_t s) {
  switch (kind) {
    case W_FP32: return launch_dd_kind<float, W_FP32>(a, grid_cap, s);
    case W_BF16: return launch_dd_kind<float, W_BF16>(a, grid_cap, s);
    case W_FP16: return launch_dd_kind<float, W_FP16>(a, grid_cap, s);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------------- K4
template <typename T>
__global__ void __launch_bounds__(256) k_dd_combine(const CombineArgs<T> a) {
  using C = typename Cx<T>::t;
  ptx::grid_dep_wait();  // launched with a programmatic dependency inside the cycle
  ptx::grid_dep_launch();
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.N) return;
  const int iy = (int)(j / a.m), ix = (int)(j - (long long)iy * a.m);
  const int4 tx = a.ctab[ix], ty = a.ctab[iy];
  const C* V = a.V + (size_t)blockIdx.y * a.nsub * a.NR;
  T sr = 0, si = 0;
  const int byl[2] = {ty.x, ty.z}, ryl[2] = {ty.y, ty.w};
  const int bxl[2] = {tx.x, tx.z}, rxl[2] = {tx.y, tx.w};
#pragma unroll
  for (int jy = 0; jy < 2; ++jy) {
    if (byl[jy] < 0) continue;
#pragma unroll
    for (int jx = 0; jx < 2; ++jx) {
      if (bxl[jx] < 0) continue;
      const C v = V[((size_t)byl[jy] * a.nb + bxl[jx]) * a.NR + ryl[jy] * a.Lu + rxl[jx]];
      sr += v.x;
      si += v.y;
    }
  }
  C* u = a.u + (size_t)blockIdx.y * a.N;
  C o;
  if (a.uin) {
    o = a.uin[(size_t)blockIdx.y * a.N + j];
    o.x += sr;
    o.y += si;
  } else if (a.accumulate) {
    o = u[j];
    o.x += sr;
    o.y += si;
  } else {
    o.x = sr;
    o.y = si;
  }
  if (a.wide) {
    double2* w = a.wide + (size_t)blockIdx.y * a.N + j;
    double2 d = a.wide_acc ? *w : make_double2(0.0, 0.0);
    d.x = a.wide_acc ? d.x + (double)o.x : (double)o.x;
    d.y = a.wide_acc ? d.y + (double)o.y : (double)o.y;
    *w = d;
  } else {
    u[j] = o;
  }
}

template <typename T>
cudaError_t launch_dd_combine(const CombineArgs<T>& a, int nrhs, cudaStream_t s) {
  dim3 grid((unsigned)((a.N + 255) / 256), nrhs);
  return launch_pdl(k_dd_combine<T>, grid, dim3(256), 0, s, 0, a);
}

template cudaError_t launch_dd_combine<double>(const CombineArgs<double>&, int, cudaStream_t);
template cudaError_t launch_dd_combine<float>(const CombineArgs<float>&, int, cudaStream_t);


// ------------------------------------------------------------------- K3 (TMA streamed)
// Persistent variant of K3: one CTA per SM walks its subdomains; the inverse
// rows of each subdomain (contiguous, chunk-major) are pulled from HBM in
// stages of up to 48 KB by one-dimensional bulk copies (cp.async.bulk, the
// TMA engine) into a ring of D shared-memory slots, each completing on its
// own mbarrier, D - 1 stages ahead of the consumers.  The next subdomain's
// gather of r is prefetched with cp.async while the current one computes.
// Every wait on an mbarrier is bounded: on timeout the CTA records a flag,
// drains its copies in flight (again bounded) and returns.
namespace {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return ptx::smem_addr(p); }
using ptx::bulk_g2s;
using ptx::mbar_init;
template <typename C>
__device__ __forceinline__ void cp_async_c(C* smem, const C* gmem) {
  if constexpr (sizeof(C) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

}  // namespace

// PK (FP32 arithmetic on 4-column BF16 / FP16 chunks, at most 4 right-hand
// sides): the gathered x is stored per chunk as [re0..re3][im0..im3] and the
// products run as paired FP32 FMAs (__ffma2_rn, two lanes per instruction):
// (wr0, wr1) * (xr0, xr1) into a real sum, (wi0, wi1) * (xi0, xi1) into a sum
// subtracted at the end, and both cross terms into the imaginary sum.
template <typename T, int KIND, int NRHS, bool PK>
__global__ void __launch_bounds__(512, 2) k_dd_stream(const DDArgs<T> a, int cps, int depth, int* err) {
  using C = typename Cx<T>::t;
  constexpr int CPC = WTraits<KIND>::CPC;
  static_assert(!PK || (std::is_same<T, float>::value && CPC == 4 && NRHS <= 4), "paired-FMA form");
  extern __shared__ __align__(128) unsigned char smraw[];
  const int NR = a.NR, NCH = a.NCH, G = a.G;
  const size_t slot_bytes = (size_t)cps * NR * 16;
  unsigned char* slots = smraw;                                             // [depth][slot_bytes]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw + depth * slot_bytes);  // [depth]
  const int XL = NCH * CPC;
  C* xs = reinterpret_cast<C*>(bars + 8);                                   // [2][NRHS][XL]
  C* red = xs + 2 * NRHS * XL;                                              // [G][NR][NRHS]
  int2* tab = reinterpret_cast<int2*>(red + (size_t)G * NR * NRHS);         // [XL]: box offset, packed (x, y, z)
  const int tid = threadIdx.x, nth = blockDim.x;
  const int rr = tid % NR, g = tid / NR;
  const int r0 = blockIdx.y * NRHS;
  const int nr = min(NRHS, a.nrhs - r0);
  const int NS = (NCH + cps - 1) / cps;
  const int nmine = (a.nsub - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int total = nmine * NS;
  const int lim = ptx::wait_limit(err, 1 << 17);  // about 1.3 s of suspending polls
  if (lim == 0) {  // waits disabled: record a timeout before any barrier or copy
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }

  int issued_hi = 0;         // thread 0: one past the last item issued
  auto issue = [&](int t) {  // thread 0 only
    if (t >= total) return;
    issued_hi = t + 1;
    const int sub = blockIdx.x + (t / NS) * gridDim.x;
    const int s = t % NS;
    const int ch0 = s * cps;
    const int nch = min(cps, NCH - ch0);
    const unsigned bytes = (unsigned)((size_t)nch * NR * 16);
    const char* src = reinterpret_cast<const char*>(a.W) + ((size_t)sub * NCH + ch0) * NR * 16;
    uint64_t* bar = bars + (t % depth);
    ptx::mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(slots + (size_t)(t % depth) * slot_bytes, src, bytes, bar);
  };
  // box-relative offsets and coordinates of the gathered columns (the same for
  // every subdomain): the per-subdomain gather does no integer division
  {
    const int L2 = a.Lw * a.Lw;
    for (int c = tid; c < XL; c += nth) {
      const int cz = c / L2, cr = c - cz * L2;
      const int cy = cr / a.Lw, cx = cr - cy * a.Lw;
      tab[c] = c < a.NC ? make_int2((cz * a.m + cy) * a.m + cx, cx | (cy << 10) | (cz << 20)) : make_int2(0, -1);
    }
  }
  auto gather = [&](int i, int buf) {
    if (i < nmine) {
      const int sub = blockIdx.x + i * gridDim.x;
      const int* bb = a.box + (size_t)sub * 12;
      const int wx = bb[2], wy = bb[3], wz = bb[9];
      const size_t base = ((size_t)bb[8] * a.m + bb[1]) * a.m + bb[0];
      C* dst = xs + (size_t)buf * NRHS * XL;
#pragma unroll
      for (int k = 0; k < NRHS; ++k) {
        const C* src = a.r + (size_t)(r0 + k) * a.N + base;
        for (int c = tid; c < XL; c += nth) {
          const int2 e = tab[c];
          const bool in = k < nr && e.y >= 0 && (e.y & 1023) < wx && ((e.y >> 10) & 1023) < wy && (e.y >> 20) < wz;
          if constexpr (PK) {  // [chunk][re0..re3, im0..im3]
            float* d = reinterpret_cast<float*>(dst + (size_t)k * XL) + (size_t)(c >> 2) * 8 + (c & 3);
            if (in) {
              const float* s2 = reinterpret_cast<const float*>(src + e.x);
              asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(d)), "l"(s2) : "memory");
              asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(d + 4)), "l"(s2 + 1) : "memory");
            } else {
              d[0] = 0.f;
              d[4] = 0.f;
            }
          } else {
            if (in) {
              cp_async_c(dst + (size_t)k * XL + c, src + e.x);
            } else {
              C z;
              z.x = 0;
              z.y = 0;
              dst[(size_t)k * XL + c] = z;
            }
          }
        }
      }
    }
    cp_commit();
  };
  __syncthreads();  // tab

  if (tid == 0) {
    for (int d = 0; d < depth; ++d) mbar_init(bars + d, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int t = 0; t < depth; ++t) issue(t);
  // the rows above are set-up data; r is the previous kernel's output
  ptx::grid_dep_wait();
  ptx::grid_dep_launch();
  gather(0, 0);
  // A wait that gives up marks `failed` (shared); every thread keeps running the
  // same loop (on possibly stale data) so the barriers stay uniform, no new
  // copies are issued, and the copies in flight are drained at the end.
  __shared__ int failed;
  if (tid == 0) failed = 0;
  int t = 0;
  for (int i = 0; i < nmine; ++i) {
    gather(i + 1, (i + 1) & 1);
    cp_wait1();
    __syncthreads();
    const C* xv = xs + (size_t)(i & 1) * NRHS * XL;
    // two accumulator sets (even / odd column of a chunk) halve the FMA chains
    T acr[2][NRHS], aci[2][NRHS];
#pragma unroll
    for (int k = 0; k < NRHS; ++k) { acr[0][k] = aci[0][k] = acr[1][k] = aci[1][k] = 0; }
    // PK: real, subtracted and imaginary pair sums; with one right-hand side
    // columns (0, 1) and (2, 3) of a chunk have their own (shorter chains),
    // with several they share one set (registers)
    constexpr int PS = NRHS == 1 ? 2 : 1;
    float2 pR[PS][NRHS], pN[PS][NRHS], pI[PS][NRHS];
#pragma unroll
    for (int k = 0; k < NRHS; ++k)
#pragma unroll
      for (int h = 0; h < PS; ++h) pR[h][k] = pN[h][k] = pI[h][k] = make_float2(0.f, 0.f);
    for (int s = 0; s < NS; ++s, ++t) {
      if (!failed && !ptx::mbar_wait_suspend(bars + (t % depth), (unsigned)((t / depth) & 1), lim)) failed = 1;
      const int ch0 = s * cps, nch = min(cps, NCH - ch0);
      const unsigned char* slot = slots + (size_t)(t % depth) * slot_bytes;
      if (g < G) {
        for (int ch = g; ch < nch; ch += G) {
          T wr[CPC], wi[CPC];
          unpack_chunk_smem<T, KIND>(slot, (size_t)ch * NR + rr, wr, wi);
          if constexpr (PK) {
            const float2 WR[2] = {make_float2(wr[0], wr[1]), make_float2(wr[2], wr[3])};
            const float2 WI[2] = {make_float2(wi[0], wi[1]), make_float2(wi[2], wi[3])};
#pragma unroll
            for (int k = 0; k < NRHS; ++k) {
              const float4* xq = reinterpret_cast<const float4*>(xv + (size_t)k * XL) + (size_t)(ch0 + ch) * 2;
              const float4 xr = xq[0], xi = xq[1];
              const float2 XR[2] = {make_float2(xr.x, xr.y), make_float2(xr.z, xr.w)};
              const float2 XI[2] = {make_float2(xi.x, xi.y), make_float2(xi.z, xi.w)};
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int q = h % PS;
                pR[q][k] = __ffma2_rn(WR[h], XR[h], pR[q][k]);
                pN[q][k] = __ffma2_rn(WI[h], XI[h], pN[q][k]);
                pI[q][k] = __ffma2_rn(WR[h], XI[h], pI[q][k]);
                pI[q][k] = __ffma2_rn(WI[h], XR[h], pI[q][k]);
              }
            }
          } else if constexpr (std::is_same<T, float>::value && CPC % 2 == 0) {
            // two complex x per 16-byte load (x rows are 16-byte aligned, chunk starts even)
#pragma unroll
            for (int k = 0; k < NRHS; ++k) {
              const float4* xq = reinterpret_cast<const float4*>(xv + (size_t)k * XL + (size_t)(ch0 + ch) * CPC);
#pragma unroll
              for (int j2 = 0; j2 < CPC / 2; ++j2) {
                const float4 x = xq[j2];
                acr[0][k] = fmadd(wr[2 * j2], x.x, acr[0][k]);
                acr[0][k] = fmadd(-wi[2 * j2], x.y, acr[0][k]);
                aci[0][k] = fmadd(wr[2 * j2], x.y, aci[0][k]);
                aci[0][k] = fmadd(wi[2 * j2], x.x, aci[0][k]);
                acr[1][k] = fmadd(wr[2 * j2 + 1], x.z, acr[1][k]);
                acr[1][k] = fmadd(-wi[2 * j2 + 1], x.w, acr[1][k]);
                aci[1][k] = fmadd(wr[2 * j2 + 1], x.w, aci[1][k]);
                aci[1][k] = fmadd(wi[2 * j2 + 1], x.z, aci[1][k]);
              }
            }
          } else {
#pragma unroll
            for (int j = 0; j < CPC; ++j) {
              const int c = (ch0 + ch) * CPC + j;
#pragma unroll
              for (int k = 0; k < NRHS; ++k) {
                const C x = xv[k * XL + c];
                acr[j & 1][k] = fmadd(wr[j], x.x, acr[j & 1][k]);
                acr[j & 1][k] = fmadd(-wi[j], x.y, acr[j & 1][k]);
                aci[j & 1][k] = fmadd(wr[j], x.y, aci[j & 1][k]);
                aci[j & 1][k] = fmadd(wi[j], x.x, aci[j & 1][k]);
              }
            }
          }
        }
      }
      __syncthreads();  // every thread is done with this slot
      if (tid == 0 && !failed) issue(t + depth);
    }
    const int sub = blockIdx.x + i * gridDim.x;
    if (g < G) {
#pragma unroll
      for (int k = 0; k < NRHS; ++k) {
        C v;
        if constexpr (PK) {
          float sr = 0.f, sn = 0.f, si = 0.f;
#pragma unroll
          for (int h = 0; h < PS; ++h) {
            sr += pR[h][k].x + pR[h][k].y;
            sn += pN[h][k].x + pN[h][k].y;
            si += pI[h][k].x + pI[h][k].y;
          }
          v.x = sr - sn;
          v.y = si;
        } else {
          v.x = acr[0][k] + acr[1][k];
          v.y = aci[0][k] + aci[1][k];
        }
        red[((size_t)g * NR + rr) * NRHS + k] = v;
      }
    }
    __syncthreads();
    if (tid < NR) {
      const T sc = a.wscale ? (T)a.wscale[sub] : (T)1;
      for (int k = 0; k < nr; ++k) {
        T sr = 0, si = 0;
        for (int gg = 0; gg < G; ++gg) {
          const C v = red[((size_t)gg * NR + tid) * NRHS + k];
          sr += v.x;
          si += v.y;
        }
        C o;
        o.x = sr * sc;
        o.y = si * sc;
        a.V[((size_t)(r0 + k) * a.nsub + sub) * NR + tid] = o;
      }
    }
  }
  cp_wait0();
  __syncthreads();
  if (tid == 0 && failed) {
    // record, then wait (bounded) for the copies that can still be in flight:
    // no item is issued before the one `depth` places earlier was consumed
    atomicExch(err, 1);
    for (int u = max(0, issued_hi - depth); u < issued_hi; ++u)
      ptx::mbar_wait_suspend(bars + (u % depth), (unsigned)((u / depth) & 1), ptx::kDrainPolls);
  }
  __syncthreads();
}

// Variant 2 of the streamed kernel: a dedicated producer warp issues the row
// copies into a ring of `depth` slots and refills a slot when every compute
// warp has released it (one mbarrier arrival per warp, no CTA barrier per
// slot); the per-subdomain synchronisation uses a named barrier over the
// compute warps only.  Three stages of up to 32 KB, two CTAs per SM: with
// per-warp release a stage is back in flight as soon as its slowest warp is
// done with it (four 24 KB stages, or 16 KB ones with three CTAs per SM, were
// slower: more stage transitions per subdomain).
template <typename T, int KIND, int NRHS>
__global__ void __launch_bounds__(512, 2) k_dd_stream2(const DDArgs<T> a, int cps, int depth, int* err) {
  using C = typename Cx<T>::t;
  constexpr int CPC = WTraits<KIND>::CPC;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int NR = a.NR, NCH = a.NCH, G = a.G;
  const size_t slot_bytes = (size_t)cps * NR * 16;
  unsigned char* slots = smraw;                                              // [depth][slot_bytes]
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw + depth * slot_bytes);  // [depth]
  uint64_t* empty = full + 8;                                                // [depth]
  const int XL = NCH * CPC;
  C* xs = reinterpret_cast<C*>(full + 16);                                   // [2][NRHS][XL]
  C* red = xs + 2 * NRHS * XL;                                               // [G][NR][NRHS]
  const int tid = threadIdx.x, lane = tid & 31;
  const int ncomp = blockDim.x - 32, nwc = ncomp / 32;
  const bool producer = tid >= ncomp;
  const int rr = tid % NR, g = tid / NR;
  const int r0 = blockIdx.y * NRHS;
  const int nr = min(NRHS, a.nrhs - r0);
  const int NS = (NCH + cps - 1) / cps;
  const int nmine = (a.nsub - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int total = nmine * NS;
  const int lim = ptx::wait_limit(err, 1 << 17);  // about 1.3 s of suspending polls
  if (lim == 0) {  // waits disabled: record a timeout before any barrier or copy
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  __shared__ volatile int failed;
  __shared__ int issued_hi;
  if (tid == 0) {
    failed = 0;
    issued_hi = 0;
    for (int d = 0; d < depth; ++d) {
      mbar_init(full + d, 1);
      mbar_init(empty + d, nwc);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (producer) {
    if (lane == 0) {
      for (int t = 0; t < total; ++t) {
        if (t >= depth && !ptx::mbar_wait_suspend(empty + (t % depth), (unsigned)(((t / depth) - 1) & 1), lim)) failed = 1;
        if (failed) break;
        const int sub = blockIdx.x + (t / NS) * gridDim.x;
        const int s = t % NS;
        const int ch0 = s * cps;
        const int nch = min(cps, NCH - ch0);
        const unsigned bytes = (unsigned)((size_t)nch * NR * 16);
        const char* src = reinterpret_cast<const char*>(a.W) + ((size_t)sub * NCH + ch0) * NR * 16;
        ptx::mbar_arrive_expect_tx(full + (t % depth), bytes);
        bulk_g2s(slots + (size_t)(t % depth) * slot_bytes, src, bytes, full + (t % depth));
        issued_hi = t + 1;
      }
    }
    __syncwarp();
  } else {
    auto gather = [&](int i, int buf) {
      if (i < nmine) {
        const int sub = blockIdx.x + i * gridDim.x;
        const int* bb = a.box + (size_t)sub * 12;
        const int ox = bb[0], oy = bb[1], wx = bb[2], wy = bb[3], oz = bb[8], wz = bb[9];
        const int L2 = a.Lw * a.Lw;
        C* dst = xs + (size_t)buf * NRHS * XL;
        for (int idx = tid; idx < NRHS * XL; idx += ncomp) {
          const int k = idx / XL, c = idx - k * XL;
          const int cz = c / L2, cr = c - cz * L2;
          const int cy = cr / a.Lw, cx = cr - cy * a.Lw;
          if (k < nr && c < a.NC && cx < wx && cy < wy && cz < wz) {
            cp_async_c(dst + idx,
                       a.r + (size_t)(r0 + k) * a.N + ((size_t)(oz + cz) * a.m + (oy + cy)) * a.m + (ox + cx));
          } else {
            C z;
            z.x = 0;
            z.y = 0;
            dst[idx] = z;
          }
        }
      }
      cp_commit();
    };
    // r is the previous kernel's output (the producer streams set-up data only)
    ptx::grid_dep_wait();
    ptx::grid_dep_launch();
    gather(0, 0);
    int t = 0;
    for (int i = 0; i < nmine; ++i) {
      gather(i + 1, (i + 1) & 1);
      cp_wait1();
      named_sync(1, ncomp);
      const C* xv = xs + (size_t)(i & 1) * NRHS * XL;
      T acr[NRHS], aci[NRHS];
#pragma unroll
      for (int k = 0; k < NRHS; ++k) { acr[k] = 0; aci[k] = 0; }
      for (int s = 0; s < NS; ++s, ++t) {
        if (!failed && !ptx::mbar_wait_suspend(full + (t % depth), (unsigned)((t / depth) & 1), lim)) failed = 1;
        const int ch0 = s * cps, nch = min(cps, NCH - ch0);
        const unsigned char* slot = slots + (size_t)(t % depth) * slot_bytes;
        if (g < G && !failed) {
          for (int ch = g; ch < nch; ch += G) {
            T wr[CPC], wi[CPC];
            unpack_chunk_smem<T, KIND>(slot, (size_t)ch * NR + rr, wr, wi);
#pragma unroll
            for (int j = 0; j < CPC; ++j) {
              const int c = (ch0 + ch) * CPC + j;
#pragma unroll
              for (int k = 0; k < NRHS; ++k) {
                const C x = xv[k * XL + c];
                acr[k] = fmadd(wr[j], x.x, acr[k]);
                acr[k] = fmadd(-wi[j], x.y, acr[k]);
                aci[k] = fmadd(wr[j], x.y, aci[k]);
                aci[k] = fmadd(wi[j], x.x, aci[k]);
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(empty + (t % depth));
      }
      const int sub = blockIdx.x + i * gridDim.x;
      if (g < G) {
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          C v;
          v.x = acr[k];
          v.y = aci[k];
          red[((size_t)g * NR + rr) * NRHS + k] = v;
        }
      }
      named_sync(1, ncomp);
      if (tid < NR) {
        const T sc = a.wscale ? (T)a.wscale[sub] : (T)1;
        for (int k = 0; k < nr; ++k) {
          T sr = 0, si = 0;
          for (int gg = 0; gg < G; ++gg) {
            const C v = red[((size_t)gg * NR + tid) * NRHS + k];
            sr += v.x;
            si += v.y;
          }
          C o;
          o.x = sr * sc;
          o.y = si * sc;
          a.V[((size_t)(r0 + k) * a.nsub + sub) * NR + tid] = o;
        }
      }
    }
    cp_wait0();
    __syncwarp();
  }
  __syncthreads();
  if (tid == ncomp && failed) {
    // record, then wait (bounded) for the copies that can still be in flight
    atomicExch(err, 1);
    for (int u = max(0, issued_hi - depth); u < issued_hi; ++u)
      ptx::mbar_wait_suspend(full + (u % depth), (unsigned)((u / depth) & 1), ptx::kDrainPolls);
  }
  __syncthreads();
}

template <typename T, int KIND, int NRHS>
static cudaError_t launch_dd_stream2_k(const DDArgs<T>& a0, int* err, int sms, cudaStream_t s) {
  using C = typename Cx<T>::t;
  constexpr int CPC = WTraits<KIND>::CPC;
  if (a0.NR > 480) return cudaErrorInvalidConfiguration;
  DDArgs<T> a = a0;  // the chunk groups shrink so that the producer warp fits in 512 threads
  a.G = std::max(1, std::min(a0.G, (480 / 32 * 32) / a0.NR));
  const int threads = ((a.NR * a.G + 31) / 32) * 32 + 32;
  if (threads > 512) return cudaErrorInvalidConfiguration;
  const int depth = 3;
  const int cps = std::max(1, (int)((32 * 1024) / ((size_t)a.NR * 16)));
  const size_t slot_bytes = (size_t)cps * a.NR * 16;
  const size_t smem = depth * slot_bytes + 16 * sizeof(uint64_t) +
                      sizeof(C) * ((size_t)2 * NRHS * a.NCH * CPC + (size_t)a.G * a.NR * NRHS);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  const int per_sm = std::max(1, std::min(3, (int)((228 * 1024) / (smem + 1024))));
  cudaError_t e = cudaFuncSetAttribute(k_dd_stream2<T, KIND, NRHS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int gx = std::min(a.nsub, per_sm * sms);
  dim3 grid(gx, (a.nrhs + NRHS - 1) / NRHS);
  return launch_pdl(k_dd_stream2<T, KIND, NRHS>, grid, dim3(threads), smem, s, 0, a, cps, depth, err);
}

template <typename T, int KIND, int NRHS, bool PK>
static cudaError_t launch_dd_stream_k(const DDArgs<T>& a, int* err, int sms, cudaStream_t s) {
  using C = typename Cx<T>::t;
  constexpr int CPC = WTraits<KIND>::CPC;
  const int threads = ((a.NR * a.G + 31) / 32) * 32;
  if (threads > 512 || a.Lw > 1023) return cudaErrorInvalidConfiguration;
  // a ring of three stages per CTA: up to 32 KB each for two CTAs per SM, or
  // (stream_small) up to 20 KB each so that three CTAs share an SM
  const int slot_target = a.stream_small ? 20 * 1024 : 32 * 1024;
  const int cps = std::max(1, (int)(slot_target / ((size_t)a.NR * 16)));
  const size_t slot_bytes = (size_t)cps * a.NR * 16;
  const size_t fixed = 8 * sizeof(uint64_t) +
                       sizeof(C) * ((size_t)2 * NRHS * a.NCH * CPC + (size_t)a.G * a.NR * NRHS) +
                       sizeof(int2) * (size_t)a.NCH * CPC;
  const int depth = 3;
  const size_t smem = depth * slot_bytes + fixed;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  const int fit = (int)((228 * 1024) / (smem + 1024));
  const int per_sm = std::max(1, std::min(a.stream_small ? 3 : 2, fit));
  cudaError_t e = cudaFuncSetAttribute(k_dd_stream<T, KIND, NRHS, PK>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int gx = std::min(a.nsub, per_sm * sms);
  dim3 grid(gx, (a.nrhs + NRHS - 1) / NRHS);
  return launch_pdl(k_dd_stream<T, KIND, NRHS, PK>, grid, dim3(threads), smem, s, 0, a, cps, depth, err);
}

template <typename T, int KIND>
static size_t dd_stream_smem(const DDArgs<T>& a, int nrhs) {
  using C = typename Cx<T>::t;
  const int cps = std::max(1, (int)((32 * 1024) / ((size_t)a.NR * 16)));
  return 3 * (size_t)cps * a.NR * 16 + 8 * sizeof(uint64_t) +
         sizeof(C) * ((size_t)2 * nrhs * a.NCH * WTraits<KIND>::CPC + (size_t)a.G * a.NR * nrhs) +
         sizeof(int2) * (size_t)a.NCH * WTraits<KIND>::CPC;
}

template <typename T, int KIND>
static cudaError_t launch_dd_stream_kind(const DDArgs<T>& a, int* err, int sms, cudaStream_t s) {
  if (a.stream_v2) {
    if (a.nrhs >= 4) return launch_dd_stream2_k<T, KIND, 4>(a, err, sms, s);
    if (a.nrhs >= 2) return launch_dd_stream2_k<T, KIND, 2>(a, err, sms, s);
    return launch_dd_stream2_k<T, KIND, 1>(a, err, sms, s);
  }
  if (a.nrhs >= 8 && dd_stream_smem<T, KIND>(a, 8) <= 227 * 1024)
    return launch_dd_stream_k<T, KIND, 8, false>(a, err, sms, s);
  constexpr bool pk = std::is_same<T, float>::value && WTraits<KIND>::CPC == 4;
  if (pk && a.stream_pk) {
    if (a.nrhs >= 4) return launch_dd_stream_k<T, KIND, 4, pk>(a, err, sms, s);
    if (a.nrhs >= 2) return launch_dd_stream_k<T, KIND, 2, pk>(a, err, sms, s);
    return launch_dd_stream_k<T, KIND, 1, pk>(a, err, sms, s);
  }
  if (a.nrhs >= 4) return launch_dd_stream_k<T, KIND, 4, false>(a, err, sms, s);
  if (a.nrhs >= 2) return launch_dd_stream_k<T, KIND, 2, false>(a, err, sms, s);
  return launch_dd_stream_k<T, KIND, 1, false>(a, err, sms, s);
}

template <>
cudaError_t launch_dd_stream<double>(const DDArgs<double>& a, int kind, int* err, int sms, cudaStream_t s) {
  if (kind != W_FP64) return cudaErrorInvalidValue;
  return launch_dd_stream_kind<double, W_FP64>(a, err, sms, s);
}
template <>
cudaError_t launch_dd_stream<float>(const DDArgs<float>& a, int kind, int* err, int sms, cudaStream_t s) {
  switch (kind) {
    case W_FP32: return launch_dd_stream_kind<float, W_FP32>(a, err, sms, s);
    case W_BF16: return launch_dd_stream_kind<float, W_BF16>(a, err, sms, s);
    case W_FP16: return launch_dd_stream_kind<float, W_FP16>(a, err, sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace th
