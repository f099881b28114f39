// K5/K6 grid transfers, K7 coarse QSFEM apply, K9/K10 vector kernels.
//
// K6 prolongation (Section 4.2): I_P u_c is, in every fine cell, the
// degree-p/2 interpolant of the coarse values at the (p/2+1)^2 coarse nodes of
// that cell; its fine nodal values are a tensor product of 1-D weights
// l^eq_b(xi_a).  K5 restriction is the transpose I_P^T (Algorithm 1).
// K7: A_q of Section 3.3 applied cell by cell: per coarse cell c the
// coefficients (d0, d1, d2) for same-node, edge-neighbour and diagonal pairs,
// plus -i k hc times the Q1 edge mass on absorbing sides.
#include "ds_math.cuh"
#include "kernels.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace th {

// -------------------------------------------------------------------- K5
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(const TransferArgs<T> a) {
  using C = typename Cx<T>::t;
  ptx::grid_dep_wait();  // launched with a programmatic dependency inside the cycle
  ptx::grid_dep_launch();
  const long long J = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= a.Nc) return;
  const int Jy = (int)(J / a.mc), Jx = (int)(J - (long long)Jy * a.mc);
  const C* r = a.in + (size_t)blockIdx.y * a.N;
  T sr = 0, si = 0;
  for (int ky = 0; ky < a.rmax; ++ky) {
    const T wy = a.rw[(size_t)Jy * a.rmax + ky];
    if (wy == (T)0) continue;
    const int iy = a.ridx[(size_t)Jy * a.rmax + ky];
    T tr = 0, ti = 0;
    for (int kx = 0; kx < a.rmax; ++kx) {
      const T wx = a.rw[(size_t)Jx * a.rmax + kx];
      const C v = r[(size_t)iy * a.m + a.ridx[(size_t)Jx * a.rmax + kx]];
      tr = fma(wx, v.x, tr);
      ti = fma(wx, v.y, ti);
    }
    sr = fma(wy, tr, sr);
    si = fma(wy, ti, si);
  }
  C o;
  o.x = sr;
  o.y = si;
  // the coarse space vanishes on Gamma_0: no restricted residual there
  if (((a.dirichlet & 1) && Jx == 0) || ((a.dirichlet & 2) && Jx == a.mc - 1) || ((a.dirichlet & 4) && Jy == 0) ||
      ((a.dirichlet & 8) && Jy == a.mc - 1)) {
    o.x = 0;
    o.y = 0;
  }
  a.out[(size_t)blockIdx.y * a.Nc + J] = o;
}

// -------------------------------------------------------------------- K6
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(const TransferArgs<T> a) {
  using C = typename Cx<T>::t;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.N) return;
  const int iy = (int)(j / a.m), ix = (int)(j - (long long)iy * a.m);
  const C* uc = a.in + (size_t)blockIdx.y * a.Nc;
  const int jx0 = a.pj0[ix], jy0 = a.pj0[iy];
  T sr = 0, si = 0;
  for (int by = 0; by <= a.q; ++by) {
    const T wy = a.pw[(size_t)iy * (a.q + 1) + by];
    if (wy == (T)0) continue;
    T tr = 0, ti = 0;
    for (int bx = 0; bx <= a.q; ++bx) {
      const T wx = a.pw[(size_t)ix * (a.q + 1) + bx];
      C v = uc[(size_t)(jy0 + by) * a.mc + jx0 + bx];
      if (a.dirichlet && coarse_on_gamma0(a.dirichlet, jx0 + bx, jy0 + by, a.mc)) {
        v.x = 0;   // the coarse space vanishes on Gamma_0
        v.y = 0;
      }
      tr = fma(wx, v.x, tr);
      ti = fma(wx, v.y, ti);
    }
    sr = fma(wy, tr, sr);
    si = fma(wy, ti, si);
  }
  C* u = a.out + (size_t)blockIdx.y * a.N;
  C o = u[j];
  o.x = fma(a.omega, sr, o.x);
  o.y = fma(a.omega, si, o.y);
  u[j] = o;
}

template <typename T>
cudaError_t launch_restrict(const TransferArgs<T>& a, int nrhs, cudaStream_t s) {
  dim3 grid((unsigned)((a.Nc + 255) / 256), nrhs);
  return launch_pdl(k_restrict<T>, grid, dim3(256), 0, s, 0, a);
}
template <typename T>
cudaError_t launch_prolong(const TransferArgs<T>& a, int nrhs, cudaStream_t s) {
  dim3 grid((unsigned)((a.N + 255) / 256), nrhs);
  k_prolong<T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_restrict<double>(const TransferArgs<double>&, int, cudaStream_t);
template cudaError_t launch_restrict<float>(const TransferArgs<float>&, int, cudaStream_t);
template cudaError_t launch_prolong<double>(const TransferArgs<double>&, int, cudaStream_t);
template cudaError_t launch_prolong<float>(const TransferArgs<float>&, int, cudaStream_t);

// -------------------------------------------------------------------- K7
template <typename C>
__device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x += a.x * b.x - a.y * b.y;
  acc.y += a.x * b.y + a.y * b.x;
}

template <typename T>
__global__ void __launch_bounds__(256) k_coarse_apply(const CoarseApplyArgs<T> a) {
  using C = typename Cx<T>::t;
  const long long J = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= a.Nc) return;
  const int Jy = (int)(J / a.mc), Jx = (int)(J - (long long)Jy * a.mc);
  const C* x = a.x + (size_t)blockIdx.y * a.Nc;
  auto dnode = [&](int ix, int iy) {
    return ((a.dirichlet & 1) && ix == 0) || ((a.dirichlet & 2) && ix == a.mc - 1) ||
           ((a.dirichlet & 4) && iy == 0) || ((a.dirichlet & 8) && iy == a.mc - 1);
  };
  if (a.dirichlet && dnode(Jx, Jy)) {  // identity row on Gamma_0
    C v = x[J];
    if (a.f) {
      const C fv = a.f[(size_t)blockIdx.y * a.Nc + J];
      v.x = fv.x - v.x;
      v.y = fv.y - v.y;
    }
    a.y[(size_t)blockIdx.y * a.Nc + J] = v;
    return;
  }
  // with Gamma_0 present the values of its nodes are left out (zero columns)
  auto xv = [&](int ix, int iy) {
    C v = x[(size_t)iy * a.mc + ix];
    if (a.dirichlet && dnode(ix, iy)) {
      v.x = 0;
      v.y = 0;
    }
    return v;
  };
  C acc;
  acc.x = 0;
  acc.y = 0;
  // cells (cx, cy) around node (Jx, Jy): cx in {Jx-1, Jx}, cy in {Jy-1, Jy}
  for (int cy = Jy - 1; cy <= Jy; ++cy) {
    if (cy < 0 || cy >= a.nc) continue;
    for (int cx = Jx - 1; cx <= Jx; ++cx) {
      if (cx < 0 || cx >= a.nc) continue;
      const C* d = a.cell + ((size_t)cy * a.nc + cx) * 3;
      const int ox = (cx == Jx) ? 1 : -1, oy = (cy == Jy) ? 1 : -1;  // direction of the other nodes
      cfma(acc, d[0], xv(Jx, Jy));
      cfma(acc, d[1], xv(Jx + ox, Jy));
      cfma(acc, d[1], xv(Jx, Jy + oy));
      cfma(acc, d[2], xv(Jx + ox, Jy + oy));
    }
  }
  // absorbing sides: rho_e (1/3 x_J + 1/6 x_neighbour) per boundary edge at J
  const T third = (T)(1.0 / 3.0), sixth = (T)(1.0 / 6.0);
  for (int s = 0; s < 4; ++s) {
    const bool xside = s < 2;
    const int fixed = xside ? Jx : Jy;
    const int along = xside ? Jy : Jx;
    if (fixed != ((s & 1) ? a.nc : 0)) continue;
    const C* rho = a.rho + (size_t)s * a.nc;
    for (int t = along - 1; t <= along; ++t) {
      if (t < 0 || t >= a.nc) continue;
      const C r = rho[t];
      const int other = (t == along) ? along + 1 : along - 1;
      C xj = x[J], xo = xside ? xv(Jx, other) : xv(other, Jy);
      C v;
      v.x = third * xj.x + sixth * xo.x;
      v.y = third * xj.y + sixth * xo.y;
      cfma(acc, r, v);
    }
  }
  if (a.f) {
    const C fv = a.f[(size_t)blockIdx.y * a.Nc + J];
    acc.x = fv.x - acc.x;
    acc.y = fv.y - acc.y;
  }
  a.y[(size_t)blockIdx.y * a.Nc + J] = acc;
}

template <typename T>
cudaError_t launch_coarse_apply(const CoarseApplyArgs<T>& a, int nrhs, cudaStream_t s) {
  dim3 grid((unsigned)((a.Nc + 255) / 256), nrhs);
  k_coarse_apply<T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_coarse_apply<double>(const CoarseApplyArgs<double>&, int, cudaStream_t);
template cudaError_t launch_coarse_apply<float>(const CoarseApplyArgs<float>&, int, cudaStream_t);

// ---------------------------------------------------------------- K10 etc.
__global__ void k_d2f(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void k_f2d(const float* __restrict__ in, double* __restrict__ out, long long n, int acc) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = acc ? out[i] + (double)in[i] : (double)in[i];
}
static unsigned vgrid(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}
__global__ void k_cadd32(float2* __restrict__ u, const float2* __restrict__ w, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float2 a = u[i];
    const float2 b = w[i];
    a.x += b.x;
    a.y += b.y;
    u[i] = a;
  }
}
cudaError_t launch_cadd32(float2* u, const float2* w, long long n, cudaStream_t s) {
  k_cadd32<<<vgrid(n), 256, 0, s>>>(u, w, n);
  return cudaGetLastError();
}
cudaError_t launch_d2f(const double* in, float* out, long long n, cudaStream_t s) {
  k_d2f<<<vgrid(n), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}
cudaError_t launch_f2d(const float* in, double* out, long long n, int accumulate, cudaStream_t s) {
  k_f2d<<<vgrid(n), 256, 0, s>>>(in, out, n, accumulate);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_zaxpy(const typename Cx<T>::t* __restrict__ x, typename Cx<T>::t* __restrict__ y, T alpha,
                        long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    auto v = y[i];
    const auto xv = x[i];
    v.x += alpha * xv.x;
    v.y += alpha * xv.y;
    y[i] = v;
  }
}
template <typename T>
cudaError_t launch_zaxpy(const typename Cx<T>::t* x, typename Cx<T>::t* y, T alpha, long long n, cudaStream_t s) {
  k_zaxpy<T><<<vgrid(n), 256, 0, s>>>(x, y, alpha, n);
  return cudaGetLastError();
}
template cudaError_t launch_zaxpy<double>(const double2*, double2*, double, long long, cudaStream_t);
template cudaError_t launch_zaxpy<float>(const float2*, float2*, float, long long, cudaStream_t);

template <typename T>
__global__ void k_zero(typename Cx<T>::t* x, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    typename Cx<T>::t z;
    z.x = 0;
    z.y = 0;
    x[i] = z;
  }
}
template <typename T>
cudaError_t launch_zero(typename Cx<T>::t* x, long long n, cudaStream_t s) {
  k_zero<T><<<vgrid(n), 256, 0, s>>>(x, n);
  return cudaGetLastError();
}
template cudaError_t launch_zero<double>(double2*, long long, cudaStream_t);
template cudaError_t launch_zero<float>(float2*, long long, cudaStream_t);

// ---------------------------------------------------------------- K9 Krylov
constexpr int kDotTile = 8;  // basis vectors per block row

int mdot_blocks(long long N) {
  long long b = (N + 1023) / 1024;
  return (int)(b > 256 ? 256 : (b < 1 ? 1 : b));
}

// part[(rhs * nvt + i) * nblk + blk] = sum over this block's range of conj(V_i) w,
// i < nvt = nv + self; index nv (self = 1) is w itself, giving ||w||^2.
__global__ void __launch_bounds__(256) k_mdot_part(const double2* __restrict__ Vb, long long vstride,
                                                   const double2* __restrict__ w, long long N, int nv, int self,
                                                   double2* __restrict__ part, int nblk) {
  const int nvt = nv + self;
  const int rhs = blockIdx.z, i0 = blockIdx.y * kDotTile;
  const int ni = min(kDotTile, nvt - i0);
  const long long chunk = (N + nblk - 1) / nblk;
  const long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  const double2* wr = w + (size_t)rhs * N;
  double ar[kDotTile], ai[kDotTile];
#pragma unroll
  for (int t = 0; t < kDotTile; ++t) { ar[t] = 0; ai[t] = 0; }
  for (long long n = lo + threadIdx.x; n < hi; n += blockDim.x) {
    const double2 wv = wr[n];
#pragma unroll
    for (int t = 0; t < kDotTile; ++t) {
      if (t < ni) {
        const double2 v = (i0 + t < nv) ? Vb[(size_t)(i0 + t) * vstride + (size_t)rhs * N + n] : wv;
        ar[t] = fmadd(v.x, wv.x, ar[t]);
        ar[t] = fmadd(v.y, wv.y, ar[t]);
        ai[t] = fmadd(v.x, wv.y, ai[t]);
        ai[t] = fmadd(-v.y, wv.x, ai[t]);
      }
    }
  }
  __shared__ double sh[2][kDotTile][256];
#pragma unroll
  for (int t = 0; t < kDotTile; ++t) {
    sh[0][t][threadIdx.x] = ar[t];
    sh[1][t][threadIdx.x] = ai[t];
  }
  __syncthreads();
  for (int stride = 128; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride) {
#pragma unroll
      for (int t = 0; t < kDotTile; ++t) {
        sh[0][t][threadIdx.x] += sh[0][t][threadIdx.x + stride];
        sh[1][t][threadIdx.x] += sh[1][t][threadIdx.x + stride];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < (unsigned)ni) {
    double2 o;
    o.x = sh[0][threadIdx.x][0];
    o.y = sh[1][threadIdx.x][0];
    part[((size_t)rhs * nvt + i0 + threadIdx.x) * nblk + blockIdx.x] = o;
  }
}

// h[idx] = sum over blocks of part[idx][b]: one warp per output, lane l takes
// blocks l, l + 32, ..., then a fixed shuffle tree (the same order every call)
__global__ void k_mdot_final(const double2* __restrict__ part, int nblk, int total, double2* __restrict__ h) {
  const int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (idx >= total) return;  // uniform over the warp
  double sr = 0, si = 0;
  for (int b = lane; b < nblk; b += 32) {
    const double2 v = part[(size_t)idx * nblk + b];
    sr += v.x;
    si += v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) {
    double2 o;
    o.x = sr;
    o.y = si;
    h[idx] = o;
  }
}

cudaError_t launch_mdot(const double2* Vbase, long long vstride, const double2* w, long long N, int nv, int self,
                        int nrhs, double2* part, double2* h, int nblk, cudaStream_t s) {
  const int nvt = nv + (self ? 1 : 0);
  dim3 grid(nblk, (nvt + kDotTile - 1) / kDotTile, nrhs);
  k_mdot_part<<<grid, 256, 0, s>>>(Vbase, vstride, w, N, nv, self ? 1 : 0, part, nblk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int total = nvt * nrhs;
  k_mdot_final<<<(total + 3) / 4, 128, 0, s>>>(part, nblk, total, h);
  return cudaGetLastError();
}

// w[rhs] += sign * sum_i h[rhs * hstride + i] V_i[rhs]
__global__ void __launch_bounds__(256) k_maxpy(const double2* __restrict__ Vb, long long vstride,
                                               const double2* __restrict__ h, int hstride, double2* __restrict__ w,
                                               long long N, int nv, double sign) {
  const int rhs = blockIdx.y;
  double2* wr = w + (size_t)rhs * N;
  const double2* hr = h + (size_t)rhs * hstride;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    double sr = 0, si = 0;
    for (int i = 0; i < nv; ++i) {
      const double2 c = hr[i];
      const double2 v = Vb[(size_t)i * vstride + (size_t)rhs * N + n];
      sr = fmadd(c.x, v.x, sr);
      sr = fmadd(-c.y, v.y, sr);
      si = fmadd(c.x, v.y, si);
      si = fmadd(c.y, v.x, si);
    }
    double2 o = wr[n];
    o.x += sign * sr;
    o.y += sign * si;
    wr[n] = o;
  }
}

cudaError_t launch_maxpy(const double2* Vbase, long long vstride, const double2* h, int hstride, double2* w,
                         long long N, int nv, int nrhs, double sign, cudaStream_t s) {
  long long b = (N + 255) / 256;
  dim3 grid((unsigned)(b > 1216 ? 1216 : b), nrhs);
  k_maxpy<<<grid, 256, 0, s>>>(Vbase, vstride, h, hstride, w, N, nv, sign);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_norm_part(const double2* __restrict__ w, long long N, double* part, int nblk) {
  const int rhs = blockIdx.y;
  const long long chunk = (N + nblk - 1) / nblk;
  const long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  const double2* wr = w + (size_t)rhs * N;
  double s = 0;
  for (long long n = lo + threadIdx.x; n < hi; n += blockDim.x) {
    const double2 v = wr[n];
    s = fmadd(v.x, v.x, s);
    s = fmadd(v.y, v.y, s);
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int stride = 128; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride) sh[threadIdx.x] += sh[threadIdx.x + stride];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)rhs * nblk + blockIdx.x] = sh[0];
}

// one warp per right-hand side, fixed lane / shuffle order (see k_mdot_final)
__global__ void k_norm_final(const double* part, int nblk, int nrhs, double* out) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= nrhs) return;
  double s = 0;
  for (int b = lane; b < nblk; b += 32) s += part[(size_t)r * nblk + b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[r] = s;
}

cudaError_t launch_norm2(const double2* w, long long N, int nrhs, double* part, double* out, int nblk,
                         cudaStream_t s) {
  dim3 grid(nblk, nrhs);
  k_norm_part<<<grid, 256, 0, s>>>(w, N, part, nblk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_norm_final<<<(nrhs + 3) / 4, 128, 0, s>>>(part, nblk, nrhs, out);
  return cudaGetLastError();
}

// ------------------------------------------------ K9 in double-single arithmetic
// The same three Gram-Schmidt kernels for the mixed form.  This GPU issues
// FP64 FMAs at 1/64 of the FP32 rate, which holds the FP64 kernels above to
// about 2.5 TB/s of vector traffic (four FMAs per complex entry and basis
// vector).  Here every FP64 operand is split exactly into two floats
// (ds_from_double: its leading 24 and next 24 significant bits); a product
// x y is formed as p = fl(x_h y_h) with its exact rounding error
// fma(x_h, y_h, -p) plus the cross terms x_h y_l + x_l y_h (Dekker; the dropped
// x_l y_l is below 2^-46 relative); a thread's running sum is a float pair
// (s, c) in which s takes the products and c the exact rounding errors of the
// additions (Knuth's two-sum) and of the products.  Each thread sums a few
// dozen products; its pair goes to FP64 for the fixed-order block and grid
// reductions of the FP64 kernels.  Relative error about 2^-44 of the sum of
// the terms' magnitudes.
// s + c in FP64 (exact while c is within 2^-29 of s's exponent range, as here)
__device__ __forceinline__ double acc_value(const dsacc& a) { return f2d_bits(a.s) + f2d_bits(a.c); }
__device__ __forceinline__ ds dneg(ds x) { return ds(-x.h, -x.l); }
// a += (s2, c2): two-sum of the leading parts, the error and c2 into the second
__device__ __forceinline__ void acc_add(dsacc& a, float s2, float c2) {
  const float t = __fadd_rn(a.s, s2);
  const float z = __fsub_rn(t, a.s);
  const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, z)), __fsub_rn(s2, z));
  a.c = __fadd_rn(a.c, __fadd_rn(c2, err));
  a.s = t;
}
// butterfly sum over the warp (every lane ends with the same pair: each step
// adds the same two pairs, and two-sum's error term is exact in either order)
__device__ __forceinline__ void acc_warp_sum(dsacc& a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, a.s, o), c2 = __shfl_xor_sync(0xffffffffu, a.c, o);
    acc_add(a, s2, c2);
  }
}

// The basis vector i of a right-hand side at entry n: FP64 (split on load) or,
// SPLIT, stored already split as (re h, re l, im h, im l) in the same 16 bytes
template <bool SPLIT>
__device__ __forceinline__ void basis_entry(const double2* __restrict__ Vb, size_t idx, ds& x, ds& y) {
  if constexpr (SPLIT) {
    const float4 q = reinterpret_cast<const float4*>(Vb)[idx];
    x = ds(q.x, q.y);
    y = ds(q.z, q.w);
  } else {
    const double2 v = Vb[idx];
    x = ds_from_double(v.x);
    y = ds_from_double(v.y);
  }
}

template <int TILE, int MINB, bool SPLIT>
__global__ void __launch_bounds__(256, MINB) k_mdot_part_ds(const double2* __restrict__ Vb, long long vstride,
                                                            const double2* __restrict__ w, long long N, int nv,
                                                            int self, double2* __restrict__ part, int nblk) {
  const int nvt = nv + self;
  const int rhs = blockIdx.z, i0 = blockIdx.y * TILE;
  const int ni = min(TILE, nvt - i0);
  const long long chunk = (N + nblk - 1) / nblk;
  const long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  const double2* wr = w + (size_t)rhs * N;
  dsacc ar[TILE], ai[TILE];
#pragma unroll
  for (int t = 0; t < TILE; ++t) {
    ar[t] = dsacc{0.f, 0.f};
    ai[t] = dsacc{0.f, 0.f};
  }
  for (long long n = lo + threadIdx.x; n < hi; n += blockDim.x) {
    const double2 wv = wr[n];
    const ds wx = ds_from_double(wv.x), wy = ds_from_double(wv.y);
#pragma unroll
    for (int t = 0; t < TILE; ++t) {
      if (t < ni) {
        ds vx = wx, vy = wy;
        if (i0 + t < nv) basis_entry<SPLIT>(Vb, (size_t)(i0 + t) * vstride + (size_t)rhs * N + n, vx, vy);
        // conj(v) w = (vx wx + vy wy) + i (vx wy - vy wx)
        acc_prod(ar[t], vx, wx);
        acc_prod(ar[t], vy, wy);
        acc_prod(ai[t], vx, wy);
        acc_prod(ai[t], dneg(vy), wx);
      }
    }
  }
  // warp sums of the pairs, then the 8 warps' values in FP64 in a fixed order
  // (only the block's ni live pairs: ni is uniform over the block)
  __shared__ double sh[2][TILE][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < TILE; ++t) {
    if (t < ni) {
      acc_warp_sum(ar[t]);
      acc_warp_sum(ai[t]);
      if (lane == 0) {
        sh[0][t][warp] = acc_value(ar[t]);
        sh[1][t][warp] = acc_value(ai[t]);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < (unsigned)ni) {
    double2 o;
    o.x = sh[0][threadIdx.x][0];
    o.y = sh[1][threadIdx.x][0];
    for (int q = 1; q < 8; ++q) {
      o.x += sh[0][threadIdx.x][q];
      o.y += sh[1][threadIdx.x][q];
    }
    part[((size_t)rhs * nvt + i0 + threadIdx.x) * nblk + blockIdx.x] = o;
  }
}

cudaError_t launch_mdot_ds(const double2* Vbase, long long vstride, const double2* w, long long N, int nv, int self,
                           int nrhs, double2* part, double2* h, int nblk, int split, cudaStream_t s) {
  const int nvt = nv + (self ? 1 : 0);
  dim3 grid(nblk, (nvt + kDotTile - 1) / kDotTile, nrhs);
  // four CTAs per SM (at most 64 registers a thread): the loads of more warps in
  // flight (measured: 0.72 of the time with the compiler's 93 registers)
  if (split)
    k_mdot_part_ds<kDotTile, 4, true><<<grid, 256, 0, s>>>(Vbase, vstride, w, N, nv, self ? 1 : 0, part, nblk);
  else
    k_mdot_part_ds<kDotTile, 4, false><<<grid, 256, 0, s>>>(Vbase, vstride, w, N, nv, self ? 1 : 0, part, nblk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int total = nvt * nrhs;
  k_mdot_final<<<(total + 3) / 4, 128, 0, s>>>(part, nblk, total, h);
  return cudaGetLastError();
}

// w[rhs] += sign * sum_i h[rhs * hstride + i] V_i[rhs]; the coefficients are
// split once per block into shared memory ([nv][re h, re l, im h, im l])
template <bool SPLIT>
__global__ void __launch_bounds__(256) k_maxpy_ds(const double2* __restrict__ Vb, long long vstride,
                                                  const double2* __restrict__ h, int hstride, double2* __restrict__ w,
                                                  long long N, int nv, double sign) {
  extern __shared__ float hsm[];
  const int rhs = blockIdx.y;
  const double2* hr = h + (size_t)rhs * hstride;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const double2 c = hr[i];
    const ds cr = ds_from_double(c.x), ci = ds_from_double(c.y);
    hsm[4 * i] = cr.h;
    hsm[4 * i + 1] = cr.l;
    hsm[4 * i + 2] = ci.h;
    hsm[4 * i + 3] = ci.l;
  }
  __syncthreads();
  double2* wr = w + (size_t)rhs * N;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    // c v = (cr vx - ci vy) + i (cr vy + ci vx); two independent sums per
    // component (even and odd i) shorten the dependent chains
    dsacc sr{0.f, 0.f}, si{0.f, 0.f}, tr{0.f, 0.f}, ti{0.f, 0.f};
    int i = 0;
    for (; i + 1 < nv; i += 2) {
      ds v0x, v0y, v1x, v1y;
      basis_entry<SPLIT>(Vb, (size_t)i * vstride + (size_t)rhs * N + n, v0x, v0y);
      basis_entry<SPLIT>(Vb, (size_t)(i + 1) * vstride + (size_t)rhs * N + n, v1x, v1y);
      const ds c0r(hsm[4 * i], hsm[4 * i + 1]), c0i(hsm[4 * i + 2], hsm[4 * i + 3]);
      const ds c1r(hsm[4 * i + 4], hsm[4 * i + 5]), c1i(hsm[4 * i + 6], hsm[4 * i + 7]);
      acc_prod(sr, c0r, v0x);
      acc_prod(tr, c1r, v1x);
      acc_prod(si, c0r, v0y);
      acc_prod(ti, c1r, v1y);
      acc_prod(sr, dneg(c0i), v0y);
      acc_prod(tr, dneg(c1i), v1y);
      acc_prod(si, c0i, v0x);
      acc_prod(ti, c1i, v1x);
    }
    if (i < nv) {
      ds vx, vy;
      basis_entry<SPLIT>(Vb, (size_t)i * vstride + (size_t)rhs * N + n, vx, vy);
      const ds cr(hsm[4 * i], hsm[4 * i + 1]), ci(hsm[4 * i + 2], hsm[4 * i + 3]);
      acc_prod(sr, cr, vx);
      acc_prod(sr, dneg(ci), vy);
      acc_prod(si, cr, vy);
      acc_prod(si, ci, vx);
    }
    acc_add(sr, tr.s, tr.c);
    acc_add(si, ti.s, ti.c);
    double2 o = wr[n];
    o.x = fmadd(sign, acc_value(sr), o.x);
    o.y = fmadd(sign, acc_value(si), o.y);
    wr[n] = o;
  }
}

cudaError_t launch_maxpy_ds(const double2* Vbase, long long vstride, const double2* h, int hstride, double2* w,
                            long long N, int nv, int nrhs, double sign, int split, cudaStream_t s) {
  long long b = (N + 255) / 256;
  dim3 grid((unsigned)(b > 1216 ? 1216 : b), nrhs);
  const size_t smem = sizeof(float) * 4 * (size_t)(nv > 0 ? nv : 1);
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  if (split)
    k_maxpy_ds<true><<<grid, 256, smem, s>>>(Vbase, vstride, h, hstride, w, N, nv, sign);
  else
    k_maxpy_ds<false><<<grid, 256, smem, s>>>(Vbase, vstride, h, hstride, w, N, nv, sign);
  return cudaGetLastError();
}

// out[rhs] = split(in[rhs] * scale[rhs]) as (re h, re l, im h, im l) (0 if the
// scale is not finite); the product in FP64, the split by ds_from_double, so
// the Gram-Schmidt kernels read exactly the numbers they would split on load.
// in and out may be the same vector.
__global__ void k_scale_split(const double2* in, float4* out, const double* __restrict__ sc, long long N) {
  const int rhs = blockIdx.y;
  const double c = sc[rhs];
  const double f = isfinite(c) ? c : 0.0;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    const double2 v = in[(size_t)rhs * N + n];
    const ds x = ds_from_double(v.x * f), y = ds_from_double(v.y * f);
    out[(size_t)rhs * N + n] = make_float4(x.h, x.l, y.h, y.l);
  }
}
cudaError_t launch_scale_split(const double2* in, double2* out, const double* inv, long long N, int nrhs,
                               cudaStream_t s) {
  long long b = (N + 255) / 256;
  dim3 grid((unsigned)(b > 1216 ? 1216 : b), nrhs);
  k_scale_split<<<grid, 256, 0, s>>>(in, reinterpret_cast<float4*>(out), inv, N);
  return cudaGetLastError();
}
// FP32 complex from the split form: h + l rounded to FP32
__global__ void k_split_to_f32(const float4* __restrict__ in, float2* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float4 q = in[i];
    out[i] = make_float2(__fadd_rn(q.x, q.y), __fadd_rn(q.z, q.w));
  }
}
cudaError_t launch_split_to_f32(const double2* in, float2* out, long long n, cudaStream_t s) {
  long long b = (n + 255) / 256;
  k_split_to_f32<<<(unsigned)(b > 152 * 32 ? 152 * 32 : b), 256, 0, s>>>(reinterpret_cast<const float4*>(in), out, n);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_norm_part_ds(const double2* __restrict__ w, long long N, double* part,
                                                      int nblk) {
  const int rhs = blockIdx.y;
  const long long chunk = (N + nblk - 1) / nblk;
  const long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  const double2* wr = w + (size_t)rhs * N;
  dsacc a{0.f, 0.f};
  for (long long n = lo + threadIdx.x; n < hi; n += blockDim.x) {
    const double2 v = wr[n];
    const ds vx = ds_from_double(v.x), vy = ds_from_double(v.y);
    acc_prod(a, vx, vx);
    acc_prod(a, vy, vy);
  }
  __shared__ double sh[8];
  acc_warp_sum(a);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc_value(a);
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = sh[0];
    for (int q = 1; q < 8; ++q) v += sh[q];
    part[(size_t)rhs * nblk + blockIdx.x] = v;
  }
}

cudaError_t launch_norm2_ds(const double2* w, long long N, int nrhs, double* part, double* out, int nblk,
                            cudaStream_t s) {
  dim3 grid(nblk, nrhs);
  k_norm_part_ds<<<grid, 256, 0, s>>>(w, N, part, nblk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_norm_final<<<(nrhs + 3) / 4, 128, 0, s>>>(part, nblk, nrhs, out);
  return cudaGetLastError();
}

__global__ void k_scale_rhs(const double2* in, double2* out, const double* __restrict__ sc,
                            long long N) {
  const int rhs = blockIdx.y;
  const double c = sc[rhs];
  const double f = isfinite(c) ? c : 0.0;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    double2 v = in[(size_t)rhs * N + n];
    v.x *= f;
    v.y *= f;
    out[(size_t)rhs * N + n] = v;
  }
}

cudaError_t launch_scale_rhs(const double2* in, double2* out, const double* inv, long long N, int nrhs,
                             cudaStream_t s) {
  long long b = (N + 255) / 256;
  dim3 grid((unsigned)(b > 1216 ? 1216 : b), nrhs);
  k_scale_rhs<<<grid, 256, 0, s>>>(in, out, inv, N);
  return cudaGetLastError();
}

}  // namespace th

namespace th {
// ------------------------------------------------- K9b Arnoldi bookkeeping
// One thread per right-hand side: column j of the Hessenberg matrix from the
// Gram-Schmidt coefficients and ||w||, the earlier Givens rotations applied, a
// new rotation, the rotated residual vector g, the scale 1/h_{j+1,j} of the next
// basis vector, and the status the host reads one iteration later.
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

__global__ void k_arnoldi(ArnoldiArgs a, int j) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.nrhs) return;
  const int m = a.m;
  double* st = a.stat + (size_t)r * 5;
  if (!a.active[r]) {
    a.scal[r] = 0.0;
    st[0] = 0.0;
    return;
  }
  const double2* h = a.h + (size_t)r * (j + 2);  // j + 1 coefficients, then ||w||^2 before the pass
  const double hn2 = a.nrm[r], hn = sqrt(hn2);
  double2* Hc = a.H + (size_t)r * (m + 1) * m + (size_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) Hc[i] = h[i];
  Hc[j + 1] = make_double2(hn, 0.0);
  a.scal[r] = (hn > 0.0 && isfinite(hn)) ? 1.0 / hn : 0.0;
  double2* cs = a.cs + (size_t)r * m;
  double2* sn = a.sn + (size_t)r * m;
  for (int i = 0; i < j; ++i) {
    const double2 x0 = Hc[i], x1 = Hc[i + 1];
    const double2 t0 = zmul(zconj(cs[i]), x0), t1 = zmul(zconj(sn[i]), x1);
    const double2 u0 = zmul(sn[i], x0), u1 = zmul(cs[i], x1);
    Hc[i] = make_double2(t0.x + t1.x, t0.y + t1.y);
    Hc[i + 1] = make_double2(u1.x - u0.x, u1.y - u0.y);
  }
  const double2 x0 = Hc[j], x1 = Hc[j + 1];
  const double den = sqrt(x0.x * x0.x + x0.y * x0.y + x1.x * x1.x + x1.y * x1.y);
  cs[j] = den > 0 ? make_double2(x0.x / den, x0.y / den) : make_double2(1.0, 0.0);
  sn[j] = den > 0 ? make_double2(x1.x / den, x1.y / den) : make_double2(0.0, 0.0);
  Hc[j] = make_double2(den, 0.0);
  Hc[j + 1] = make_double2(0.0, 0.0);
  double2* g = a.g + (size_t)r * (m + 1);
  const double2 gj = g[j];
  const double2 gn = zmul(sn[j], gj);
  g[j + 1] = make_double2(-gn.x, -gn.y);
  g[j] = zmul(zconj(cs[j]), gj);
  const double res = sqrt(g[j + 1].x * g[j + 1].x + g[j + 1].y * g[j + 1].y);
  const bool conv = res <= a.tol * a.fn[r] || hn == 0.0;
  // status: [0] 1 while active after this step, [1] last step done (1-based), [2] 1 after severe
  // cancellation in the single Gram-Schmidt pass, [3] 1 if ||w|| is not finite, [4] the
  // residual estimate |g_{j+1}| / ||f||
  st[0] = conv ? 0.0 : 1.0;
  st[1] = (double)(j + 1);
  st[2] = (hn2 < 1e-4 * h[j + 1].x) ? 1.0 : 0.0;
  st[3] = isfinite(hn) ? 0.0 : 1.0;
  st[4] = a.fn[r] > 0.0 ? res / a.fn[r] : 0.0;
  if (conv) a.active[r] = 0;
}

cudaError_t launch_arnoldi(const ArnoldiArgs& a, int j, cudaStream_t s) {
  k_arnoldi<<<(a.nrhs + 63) / 64, 64, 0, s>>>(a, j);
  return cudaGetLastError();
}
}  // namespace th
