// Three-dimensional kernels (unit cube, Q2 elements, fitted 27-point coarse
// operator).  Same steps as the 2-D path (Algorithms 1 and 2):
//   K1-3D  k_fine3_cells + k_fine3_gather: y = A u or f - A u (Section 3.1,
//          Eq. bilin_form in 3-D: h (K M M + M K M + M M K) - c h^3 M M M per
//          cell, -i k h^2 M M on absorbing faces).  Pass 1 computes every
//          cell's 27 local outputs once (one warp per cell, lane = local node,
//          the three 1-D contractions by warp shuffles) into [cell][32];
//          pass 2 sums, per node, its (at most 8) cells in a fixed order.
//   K4-3D  k_dd_combine3: u_j (+)= sum of the (at most 8) subdomain rows holding j.
//   K5/K6  k_restrict3 / k_prolong3: tensor products of the 1-D transfer tables.
//   K7-3D  k_coarse_apply3: y_c = A_q x_c with 4 pair weights per coarse cell.
//   K8-3D  k_sweep3_couple + k_sweep3_gemv: block forward / backward sweep over
//          the z-slices of the coarse grid, one launch pair per slice.
#include "ds_math.cuh"
#include "kernels.h"

namespace th {

template <typename C>
__device__ __forceinline__ void c_fma(C& acc, C a, C b) {
  cmadd(acc, a, b);
}
template <typename T>
__device__ __forceinline__ typename Cx<T>::t shfl_c(typename Cx<T>::t v, int src) {
  typename Cx<T>::t o;
  if constexpr (std::is_same<T, ds>::value) {
    o.x = ds(__shfl_sync(0xffffffffu, v.x.h, src), __shfl_sync(0xffffffffu, v.x.l, src));
    o.y = ds(__shfl_sync(0xffffffffu, v.y.h, src), __shfl_sync(0xffffffffu, v.y.l, src));
  } else {
    o.x = __shfl_sync(0xffffffffu, v.x, src);
    o.y = __shfl_sync(0xffffffffu, v.y, src);
  }
  return o;
}

// ------------------------------------------------------------ K1-3D pass 1
template <typename T>
__global__ void __launch_bounds__(256) k_fine3_cells(const Fine3Args<T> a) {
  using C = typename Cx<T>::t;
  const int lane = threadIdx.x & 31;
  const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (cell >= a.ncell) return;  // uniform over the warp
  const int n = a.n, m = a.m;
  const int cz = (int)(cell / ((long long)n * n)), cy = (int)((cell / n) % n), cx = (int)(cell % n);
  const bool act = lane < 27;
  const int l = act ? lane : 0;
  const int az = l / 9, ay = (l / 3) % 3, ax = l % 3;
  C U;
  U.x = 0;
  U.y = 0;
  if (act) U = NodeIO<T>::ld(a.u, (size_t)blockIdx.y * a.N + ((size_t)(2 * cz + az) * m + (2 * cy + ay)) * m + (2 * cx + ax));
  // x: XM = M_x U, XK = K_x U
  C XM, XK;
  XM.x = XM.y = XK.x = XK.y = 0;
  const int bx0 = l - ax;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const C v = shfl_c<T>(U, bx0 + b);
    XM.x += a.M[ax * 3 + b] * v.x;
    XM.y += a.M[ax * 3 + b] * v.y;
    XK.x += a.K[ax * 3 + b] * v.x;
    XK.y += a.K[ax * 3 + b] * v.y;
  }
  // y: A = M_y M_x U, B = K_y M_x U, Cc = M_y K_x U
  C A, B, Cc;
  A.x = A.y = B.x = B.y = Cc.x = Cc.y = 0;
  const int by0 = l - ay * 3;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const C vm = shfl_c<T>(XM, by0 + 3 * b), vk = shfl_c<T>(XK, by0 + 3 * b);
    const T my = a.M[ay * 3 + b], ky = a.K[ay * 3 + b];
    A.x += my * vm.x;
    A.y += my * vm.y;
    B.x += ky * vm.x;
    B.y += ky * vm.y;
    Cc.x += my * vk.x;
    Cc.y += my * vk.y;
  }
  // z: Y = K_z (h A) + M_z (h (B + Cc) + m_e h^3 A), m_e = -(k^2 (1 + i alpha) + i eps)
  const T kk = a.kc[cell], ee = a.ec[cell], h = a.h, h3 = h * h * h;
  const T mr = -kk * kk * h3, mi = -(a.alpha * kk * kk + ee) * h3;
  C W1, W2;
  W1.x = h * A.x;
  W1.y = h * A.y;
  W2.x = h * (B.x + Cc.x) + (mr * A.x - mi * A.y);
  W2.y = h * (B.y + Cc.y) + (mr * A.y + mi * A.x);
  C Y;
  Y.x = Y.y = 0;
  const int bz0 = l - az * 9;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const C v1 = shfl_c<T>(W1, bz0 + 9 * b), v2 = shfl_c<T>(W2, bz0 + 9 * b);
    const T kz = a.K[az * 3 + b], mz = a.M[az * 3 + b];
    Y.x = fmadd(kz, v1.x, Y.x);
    Y.x = fmadd(mz, v2.x, Y.x);
    Y.y = fmadd(kz, v1.y, Y.y);
    Y.y = fmadd(mz, v2.y, Y.y);
  }
  // absorbing faces of the domain: -i k h^2 (M M) on the face's nodes
  const bool face[6] = {cx == 0, cx == n - 1, cy == 0, cy == n - 1, cz == 0, cz == n - 1};
  int touch = 0;
#pragma unroll
  for (int s = 0; s < 6; ++s)
    if (face[s] && ((a.robin >> s) & 1)) touch |= 1 << s;
  if (touch) {  // uniform over the warp
    const T kh2 = kk * h * h;
    // F_z = M_y M_x U = A; F_y = M_z M_x U; F_x = M_z M_y U
    C Fy, UY, Fx;
    Fy.x = Fy.y = UY.x = UY.y = Fx.x = Fx.y = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const C vm = shfl_c<T>(XM, bz0 + 9 * b);
      Fy.x += a.M[az * 3 + b] * vm.x;
      Fy.y += a.M[az * 3 + b] * vm.y;
      const C vu = shfl_c<T>(U, by0 + 3 * b);
      UY.x += a.M[ay * 3 + b] * vu.x;
      UY.y += a.M[ay * 3 + b] * vu.y;
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const C v = shfl_c<T>(UY, bz0 + 9 * b);
      Fx.x += a.M[az * 3 + b] * v.x;
      Fx.y += a.M[az * 3 + b] * v.y;
    }
    auto add = [&](const C& F) {  // Y += -i k h^2 F
      Y.x += kh2 * F.y;
      Y.y -= kh2 * F.x;
    };
    if (((touch >> 0) & 1) && ax == 0) add(Fx);
    if (((touch >> 1) & 1) && ax == 2) add(Fx);
    if (((touch >> 2) & 1) && ay == 0) add(Fy);
    if (((touch >> 3) & 1) && ay == 2) add(Fy);
    if (((touch >> 4) & 1) && az == 0) add(A);
    if (((touch >> 5) & 1) && az == 2) add(A);
  }
  if (act) a.ycell[((size_t)blockIdx.y * a.ncell + cell) * 32 + lane] = Y;
}

// ------------------------------------------------------------ K1-3D pass 2
template <typename T>
__global__ void __launch_bounds__(256) k_fine3_gather(const Fine3Args<T> a) {
  using C = typename Cx<T>::t;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.N) return;
  const int m = a.m, n = a.n;
  const int iz = (int)(j / ((long long)m * m)), iy = (int)((j / m) % m), ix = (int)(j % m);
  int cz[2], lz[2], cy[2], ly[2], cxx[2], lx[2];
  int nz = 0, ny = 0, nx = 0;
  auto cells = [&](int i, int* c, int* lo, int& cnt) {
    if (i & 1) {
      c[cnt] = i >> 1;
      lo[cnt++] = 1;
    } else {
      if ((i >> 1) - 1 >= 0) { c[cnt] = (i >> 1) - 1; lo[cnt++] = 2; }
      if ((i >> 1) < n) { c[cnt] = i >> 1; lo[cnt++] = 0; }
    }
  };
  cells(iz, cz, lz, nz);
  cells(iy, cy, ly, ny);
  cells(ix, cxx, lx, nx);
  const C* yc = a.ycell + (size_t)blockIdx.y * a.ncell * 32;
  T sr = 0, si = 0;
  for (int p = 0; p < nz; ++p)
    for (int q = 0; q < ny; ++q)
      for (int r = 0; r < nx; ++r) {
        const C v = yc[(((size_t)cz[p] * n + cy[q]) * n + cxx[r]) * 32 + lz[p] * 9 + ly[q] * 3 + lx[r]];
        sr += v.x;
        si += v.y;
      }
  C out;
  if (a.residual) {
    const C f = NodeIO<T>::ld(a.f, (size_t)blockIdx.y * a.N + j);
    out.x = f.x - sr;
    out.y = f.y - si;
  } else {
    out.x = sr;
    out.y = si;
  }
  NodeIO<T>::st(a.y, (size_t)blockIdx.y * a.N + j, out);
}

template <typename T>
cudaError_t launch_fine3(const Fine3Args<T>& a, int nrhs, cudaStream_t s) {
  dim3 g1((unsigned)((a.ncell * 32 + 255) / 256), nrhs);
  k_fine3_cells<T><<<g1, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 g2((unsigned)((a.N + 255) / 256), nrhs);
  k_fine3_gather<T><<<g2, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_fine3<double>(const Fine3Args<double>&, int, cudaStream_t);
template cudaError_t launch_fine3<float>(const Fine3Args<float>&, int, cudaStream_t);
template cudaError_t launch_fine3<ds>(const Fine3Args<ds>&, int, cudaStream_t);

// ------------------------------------------------------------ K4-3D combine
template <typename T>
__global__ void __launch_bounds__(256) k_dd_combine3(const CombineArgs<T> a) {
  using C = typename Cx<T>::t;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.N) return;
  const int m = a.m;
  const int iz = (int)(j / ((long long)m * m)), iy = (int)((j / m) % m), ix = (int)(j % m);
  const int4 tz = a.ctab[iz], ty = a.ctab[iy], tx = a.ctab[ix];
  const int bz[2] = {tz.x, tz.z}, rz[2] = {tz.y, tz.w};
  const int byl[2] = {ty.x, ty.z}, ryl[2] = {ty.y, ty.w};
  const int bxl[2] = {tx.x, tx.z}, rxl[2] = {tx.y, tx.w};
  const C* V = a.V + (size_t)blockIdx.y * a.nsub * a.NR;
  T sr = 0, si = 0;
  for (int pz = 0; pz < 2; ++pz) {
    if (bz[pz] < 0) continue;
    for (int py = 0; py < 2; ++py) {
      if (byl[py] < 0) continue;
      for (int px = 0; px < 2; ++px) {
        if (bxl[px] < 0) continue;
        const int sub = (bz[pz] * a.nb + byl[py]) * a.nb + bxl[px];
        const int row = (rz[pz] * a.Lu + ryl[py]) * a.Lu + rxl[px];
        const C v = V[(size_t)sub * a.NR + row];
        sr += v.x;
        si += v.y;
      }
    }
  }
  C* u = a.u + (size_t)blockIdx.y * a.N;
  C o;
  if (a.accumulate) {
    o = u[j];
    o.x += sr;
    o.y += si;
  } else {
    o.x = sr;
    o.y = si;
  }
  u[j] = o;
}

template <typename T>
cudaError_t launch_dd_combine3(const CombineArgs<T>& a, int nrhs, cudaStream_t s) {
  dim3 grid((unsigned)((a.N + 255) / 256), nrhs);
  k_dd_combine3<T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_dd_combine3<double>(const CombineArgs<double>&, int, cudaStream_t);
template cudaError_t launch_dd_combine3<float>(const CombineArgs<float>&, int, cudaStream_t);

// ------------------------------------------------------------ K5/K6 3-D
template <typename T>
__global__ void __launch_bounds__(256) k_restrict3(const TransferArgs<T> a) {
  using C = typename Cx<T>::t;
  const long long J = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= a.Nc) return;
  const int mc = a.mc, m = a.m, R = a.rmax;
  const int Jz = (int)(J / ((long long)mc * mc)), Jy = (int)((J / mc) % mc), Jx = (int)(J % mc);
  const C* r = a.in + (size_t)blockIdx.y * a.N;
  T sr = 0, si = 0;
  for (int kz = 0; kz < R; ++kz) {
    const T wz = a.rw[(size_t)Jz * R + kz];
    if (wz == (T)0) continue;
    const int iz = a.ridx[(size_t)Jz * R + kz];
    for (int ky = 0; ky < R; ++ky) {
      const T wy = a.rw[(size_t)Jy * R + ky];
      if (wy == (T)0) continue;
      const int iy = a.ridx[(size_t)Jy * R + ky];
      T tr = 0, ti = 0;
      for (int kx = 0; kx < R; ++kx) {
        const T wx = a.rw[(size_t)Jx * R + kx];
        const C v = r[((size_t)iz * m + iy) * m + a.ridx[(size_t)Jx * R + kx]];
        tr += wx * v.x;
        ti += wx * v.y;
      }
      sr += wz * wy * tr;
      si += wz * wy * ti;
    }
  }
  C o;
  o.x = sr;
  o.y = si;
  a.out[(size_t)blockIdx.y * a.Nc + J] = o;
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong3(const TransferArgs<T> a) {
  using C = typename Cx<T>::t;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.N) return;
  const int m = a.m, mc = a.mc, q = a.q;
  const int iz = (int)(j / ((long long)m * m)), iy = (int)((j / m) % m), ix = (int)(j % m);
  const C* uc = a.in + (size_t)blockIdx.y * a.Nc;
  const int jz0 = a.pj0[iz], jy0 = a.pj0[iy], jx0 = a.pj0[ix];
  T sr = 0, si = 0;
  for (int bz = 0; bz <= q; ++bz) {
    const T wz = a.pw[(size_t)iz * (q + 1) + bz];
    if (wz == (T)0) continue;
    for (int by = 0; by <= q; ++by) {
      const T wy = a.pw[(size_t)iy * (q + 1) + by];
      if (wy == (T)0) continue;
      T tr = 0, ti = 0;
      for (int bx = 0; bx <= q; ++bx) {
        const T wx = a.pw[(size_t)ix * (q + 1) + bx];
        const C v = uc[((size_t)(jz0 + bz) * mc + (jy0 + by)) * mc + jx0 + bx];
        tr += wx * v.x;
        ti += wx * v.y;
      }
      sr += wz * wy * tr;
      si += wz * wy * ti;
    }
  }
  C* u = a.out + (size_t)blockIdx.y * a.N;
  C o = u[j];
  o.x += a.omega * sr;
  o.y += a.omega * si;
  u[j] = o;
}

template <typename T>
cudaError_t launch_restrict3(const TransferArgs<T>& a, int nrhs, cudaStream_t s) {
  dim3 grid((unsigned)((a.Nc + 255) / 256), nrhs);
  k_restrict3<T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_prolong3(const TransferArgs<T>& a, int nrhs, cudaStream_t s) {
  dim3 grid((unsigned)((a.N + 255) / 256), nrhs);
  k_prolong3<T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_restrict3<double>(const TransferArgs<double>&, int, cudaStream_t);
template cudaError_t launch_restrict3<float>(const TransferArgs<float>&, int, cudaStream_t);
template cudaError_t launch_prolong3<double>(const TransferArgs<double>&, int, cudaStream_t);
template cudaError_t launch_prolong3<float>(const TransferArgs<float>&, int, cudaStream_t);

// ------------------------------------------------------------ K7-3D
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_apply3(const CoarseApplyArgs<T> a) {
  using C = typename Cx<T>::t;
  const long long J = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= a.Nc) return;
  const int mc = a.mc, nc = a.nc;
  const int Jv[3] = {(int)(J % mc), (int)((J / mc) % mc), (int)(J / ((long long)mc * mc))};  // x, y, z
  const C* x = a.x + (size_t)blockIdx.y * a.Nc;
  auto X = [&](int vx, int vy, int vz) { return x[((size_t)vz * mc + vy) * mc + vx]; };
  C acc;
  acc.x = 0;
  acc.y = 0;
  for (int cz = Jv[2] - 1; cz <= Jv[2]; ++cz) {
    if (cz < 0 || cz >= nc) continue;
    for (int cy = Jv[1] - 1; cy <= Jv[1]; ++cy) {
      if (cy < 0 || cy >= nc) continue;
      for (int cx = Jv[0] - 1; cx <= Jv[0]; ++cx) {
        if (cx < 0 || cx >= nc) continue;
        const C* d = a.cell + (((size_t)cz * nc + cy) * nc + cx) * 4;
        const int vz = Jv[2] - cz, vy = Jv[1] - cy, vx = Jv[0] - cx;
        for (int wz = 0; wz < 2; ++wz)
          for (int wy = 0; wy < 2; ++wy)
            for (int wx = 0; wx < 2; ++wx) {
              const int nd = (wz != vz) + (wy != vy) + (wx != vx);
              c_fma(acc, d[nd], X(cx + wx, cy + wy, cz + wz));
            }
      }
    }
  }
  // absorbing faces: rho (Q1 face mass) per face cell at J
  const T Mq[2][2] = {{(T)(1.0 / 3.0), (T)(1.0 / 6.0)}, {(T)(1.0 / 6.0), (T)(1.0 / 3.0)}};
  for (int s = 0; s < 6; ++s) {
    const int ax = s / 2, end = s % 2;
    if (Jv[ax] != (end ? nc : 0)) continue;
    const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
    for (int f2 = Jv[a2] - 1; f2 <= Jv[a2]; ++f2) {
      if (f2 < 0 || f2 >= nc) continue;
      for (int f1 = Jv[a1] - 1; f1 <= Jv[a1]; ++f1) {
        if (f1 < 0 || f1 >= nc) continue;
        const C rv = a.rho[((size_t)s * nc + f2) * nc + f1];
        const int v1 = Jv[a1] - f1, v2 = Jv[a2] - f2;
        for (int w2 = 0; w2 < 2; ++w2)
          for (int w1 = 0; w1 < 2; ++w1) {
            int v[3];
            v[ax] = Jv[ax];
            v[a1] = f1 + w1;
            v[a2] = f2 + w2;
            const T wgt = Mq[v1][w1] * Mq[v2][w2];
            C r;
            r.x = rv.x * wgt;
            r.y = rv.y * wgt;
            c_fma(acc, r, X(v[0], v[1], v[2]));
          }
      }
    }
  }
  a.y[(size_t)blockIdx.y * a.Nc + J] = acc;
}

template <typename T>
cudaError_t launch_coarse_apply3(const CoarseApplyArgs<T>& a, int nrhs, cudaStream_t s) {
  dim3 grid((unsigned)((a.Nc + 255) / 256), nrhs);
  k_coarse_apply3<T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_coarse_apply3<double>(const CoarseApplyArgs<double>&, int, cudaStream_t);
template cudaError_t launch_coarse_apply3<float>(const CoarseApplyArgs<float>&, int, cudaStream_t);

// ------------------------------------------------------------ K8-3D
// Forward: z_j = G_j (b_j - C_{j-1}^T z_{j-1}); backward: y_j = z_j - G_j C_j y_{j+1}.
// k_sweep3_couple forms the vector G_j multiplies (t), k_sweep3_gemv applies
// G_j (one warp per row, NB right-hand sides per warp).
template <typename T>
__global__ void __launch_bounds__(256) k_sweep3_couple(const Sweep3Args<T> a, int j, int backward) {
  using C = typename Cx<T>::t;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.mb) return;
  const int rhs = blockIdx.y;
  const int mc = a.mc, y = b / mc, xx = b % mc;
  const C* X = a.x + (size_t)rhs * a.Nc;
  C acc;
  acc.x = 0;
  acc.y = 0;
  const int nj = backward ? j + 1 : j - 1;  // the slice the coupling reads
  if (nj >= 0 && nj < mc) {
    const C* cf = (backward ? a.up : a.dn) + ((size_t)j * a.mb + b) * 9;
    const C* src = X + (size_t)nj * a.mb;
    for (int dy = -1; dy <= 1; ++dy) {
      if (y + dy < 0 || y + dy >= mc) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        if (xx + dx < 0 || xx + dx >= mc) continue;
        c_fma(acc, cf[(dy + 1) * 3 + dx + 1], src[(y + dy) * mc + xx + dx]);
      }
    }
  }
  C t;
  if (backward) {
    t = acc;
  } else {
    const C bj = a.b[(size_t)rhs * a.Nc + (size_t)j * a.mb + b];
    t.x = bj.x - acc.x;
    t.y = bj.y - acc.y;
  }
  a.t[(size_t)rhs * a.mb + b] = t;
}

template <typename T, int NB>
__global__ void __launch_bounds__(512) k_sweep3_gemv(const Sweep3Args<T> a, int j, int backward) {
  using C = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char sw_sm[];
  C* ts = reinterpret_cast<C*>(sw_sm);  // [NB][mb]: this tile's coupled right-hand sides
  const int lane = threadIdx.x & 31;
  const int r0 = blockIdx.y * NB, nb = min(NB, a.nrhs - r0);
  for (int i = threadIdx.x; i < NB * a.mb; i += blockDim.x) {
    const int r = i / a.mb, c = i - r * a.mb;
    C v;
    v.x = 0;
    v.y = 0;
    if (r < nb) v = a.t[(size_t)(r0 + r) * a.mb + c];
    ts[i] = v;
  }
  __syncthreads();
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= a.mb) return;
  const C* g = a.G + ((size_t)j * a.mb + row) * a.mb;
  C acc[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    acc[r].x = 0;
    acc[r].y = 0;
  }
#pragma unroll 4
  for (int c = lane; c < a.mb; c += 32) {
    const C gv = g[c];
#pragma unroll
    for (int r = 0; r < NB; ++r) c_fma(acc[r], gv, ts[r * a.mb + c]);
  }
#pragma unroll
  for (int r = 0; r < NB; ++r) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, o);
      acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, o);
    }
  }
  if (lane < nb) {
    C v = acc[0];
#pragma unroll
    for (int r = 1; r < NB; ++r)
      if (lane == r) v = acc[r];
    C* xo = a.x + (size_t)(r0 + lane) * a.Nc + (size_t)j * a.mb + row;
    if (backward) {
      C z = *xo;
      z.x -= v.x;
      z.y -= v.y;
      *xo = z;
    } else {
      *xo = v;
    }
  }
}

// NB right-hand sides per warp: every pivot block is read once per tile of NB
template <typename T, int NB>
static cudaError_t launch_sweep3_nb(const Sweep3Args<T>& a, cudaStream_t s) {
  using C = typename Cx<T>::t;
  const size_t smem = sizeof(C) * (size_t)NB * a.mb;  // the tile's coupled vectors, staged per CTA
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_sweep3_gemv<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 gc((unsigned)((a.mb + 255) / 256), a.nrhs);
  const dim3 gg((unsigned)(((long long)a.mb * 32 + 511) / 512), (a.nrhs + NB - 1) / NB);
  for (int j = 0; j < a.mc; ++j) {
    k_sweep3_couple<T><<<gc, 256, 0, s>>>(a, j, 0);
    k_sweep3_gemv<T, NB><<<gg, 512, smem, s>>>(a, j, 0);
  }
  for (int j = a.mc - 2; j >= 0; --j) {
    k_sweep3_couple<T><<<gc, 256, 0, s>>>(a, j, 1);
    k_sweep3_gemv<T, NB><<<gg, 512, smem, s>>>(a, j, 1);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sweep3(const Sweep3Args<T>& a, cudaStream_t s) {
  // the blocks stay in L2 across the rhs tiles of one step: narrower tiles give more warps
  if (a.nrhs > 4) return launch_sweep3_nb<T, 2>(a, s);
  return launch_sweep3_nb<T, 4>(a, s);
}
template cudaError_t launch_sweep3<double>(const Sweep3Args<double>&, cudaStream_t);
template cudaError_t launch_sweep3<float>(const Sweep3Args<float>&, cudaStream_t);

}  // namespace th
