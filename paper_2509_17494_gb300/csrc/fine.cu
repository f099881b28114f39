// K1/K2: matrix-free, sum-factorised apply of the fine Q_p operators A and A_s
// (Section 3.1, Eq. bilin_form; the shifted coefficient of Section 4.1), fused
// with the residual r = f - A u.
//
// Per cell e with local nodal values U[ay][ax]:
//   Y = M T2 + (K + m_e M) T1,   T1 = U M^T,  T2 = U K^T (contractions along x),
//   m_e = -(k_e^2 (1 + i alpha) + i eps_e) h^2,
// plus -i k_e h M (1-D) on the nodes of absorbing boundary sides.
// A CTA owns a TC x TC tile of cells and the nodes [cx0 p, (cx0+TC) p) of it
// (the last tile also owns the closing node).  It stages the nodal values of
// its cells and of the halo cell layer below/left of the tile in shared
// memory, computes every cell matrix-vector product there, and sums the
// contributions of the 1, 2 or 4 cells around each owned node in a fixed
// order, so the result is bitwise deterministic.
#include <type_traits>

#include "ds_math.cuh"
#include "kernels.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace th {

template <typename C, typename T>
__device__ __forceinline__ C cmul(C a, T br, T bi) {
  C r;
  r.x = a.x * br - a.y * bi;
  r.y = a.x * bi + a.y * br;
  return r;
}

// The RAS-like average at node (gx, gy) of this CTA's right-hand side: the sum
// of the V entries of the (at most 2 x 2) U boxes holding the node, in the
// order of k_dd_combine, so the fused cycle is bitwise the unfused one.
template <typename T>
__device__ __forceinline__ typename Cx<T>::t combine_at(const FineArgs<T>& a, int gx, int gy) {
  using C = typename Cx<T>::t;
  const int4 tx = a.ctab[gx], ty = a.ctab[gy];
  const C* V = a.V + (size_t)blockIdx.z * a.nsub * a.NR;
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
  C o;
  o.x = sr;
  o.y = si;
  return o;
}

// uin + omega I_P uc at node (gx, gy), in the order of k_prolong
template <typename T>
__device__ __forceinline__ typename Cx<T>::t prolong_at(const FineArgs<T>& a, int gx, int gy) {
  using C = typename Cx<T>::t;
  const C* uc = a.uc + (size_t)blockIdx.z * a.Nc;
  const int jx0 = a.pj0[gx], jy0 = a.pj0[gy];
  T sr = 0, si = 0;
  for (int by = 0; by <= a.q; ++by) {
    const T wy = a.pw[(size_t)gy * (a.q + 1) + by];
    if (wy == (T)0) continue;
    T tr = 0, ti = 0;
    for (int bx = 0; bx <= a.q; ++bx) {
      const T wx = a.pw[(size_t)gx * (a.q + 1) + bx];
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
  C o = a.uin[(size_t)blockIdx.z * a.N + (size_t)gy * a.m + gx];
  o.x = fma(a.omega, sr, o.x);
  o.y = fma(a.omega, si, o.y);
  return o;
}

template <int P, int TC, typename T>
__global__ void __launch_bounds__(TC >= 8 ? 256 : 128) k_fine_apply(const FineArgs<T> a) {
  using C = typename Cx<T>::t;
  constexpr int NP = P + 1, E = TC + 1, UT = E * P + 1, CELLS = E * E;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* su = reinterpret_cast<C*>(smraw);
  C* s1 = su + UT * UT;
  C* s2 = s1 + CELLS * NP * NP;
  constexpr int WO = TC * P + 1;                       // owned nodes per direction, at most
  C* sf = s2 + CELLS * NP * NP;                        // [WO * WO] right-hand side at the owned nodes
  T* skc = reinterpret_cast<T*>(sf + WO * WO);         // [CELLS] k, then eps, of the tile's cells
  T* sec = skc + CELLS;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int cx0 = blockIdx.x * TC, cy0 = blockIdx.y * TC;
  const int ex0 = cx0 - 1, ey0 = cy0 - 1;
  const size_t roff = (size_t)blockIdx.z * a.N;
  const C* u = a.u + roff;
  // owned nodes (phase 3)
  const int ncx = min(TC, a.n - cx0), ncy = min(TC, a.n - cy0);
  const int wx = ncx * P + ((cx0 + ncx == a.n) ? 1 : 0);
  const int wy = ncy * P + ((cy0 + ncy == a.n) ? 1 : 0);
  ptx::grid_dep_wait();  // launched with a programmatic dependency inside the cycle
  ptx::grid_dep_launch();

  // Every global load of the tile is issued here, before the first barrier, so
  // the CTA waits for memory once: its nodal values, its cells' coefficients
  // and (residual form) the right-hand side at its owned nodes.
  for (int i = tid; i < UT * UT; i += nth) {
    const int iy = i / UT, ix = i - iy * UT;
    const int gx = ex0 * P + ix, gy = ey0 * P + iy;
    C v;
    v.x = 0;
    v.y = 0;
    const bool on_d = ((a.dirichlet & 1) && gx == 0) || ((a.dirichlet & 2) && gx == a.m - 1) ||
                      ((a.dirichlet & 4) && gy == 0) || ((a.dirichlet & 8) && gy == a.m - 1);
    if (gx >= 0 && gx < a.m && gy >= 0 && gy < a.m && !on_d) {  // Gamma_0 nodes: zero columns
      if constexpr (std::is_same<T, ds>::value) {
        v = NodeIO<T>::ld(u, (size_t)gy * a.m + gx);
      } else {
        if (a.src == 1) {
          v = combine_at(a, gx, gy);
        } else if (a.src == 2) {
          v = prolong_at(a, gx, gy);
        } else {
          v = NodeIO<T>::ld(u, (size_t)gy * a.m + gx);
        }
      }
    }
    su[i] = v;
  }
  for (int e = tid; e < CELLS; e += nth) {
    const int ecy = e / E, ecx = e - ecy * E;
    const int gcx = ex0 + ecx, gcy = ey0 + ecy;
    if (gcx >= 0 && gcx < a.n && gcy >= 0 && gcy < a.n) {
      const size_t cell = (size_t)gcy * a.n + gcx;
      skc[e] = a.kc[cell];
      sec[e] = a.ec[cell];
    }
  }
  if (a.f)
    for (int i = tid; i < wx * wy; i += nth) {
      const int ly = i / wx, lx = i - ly * wx;
      sf[i] = NodeIO<T>::ld(a.f, roff + (size_t)(cy0 * P + ly) * a.m + (cx0 * P + lx));
    }
  __syncthreads();

  // phase 1: x-contractions of every row of every (extended) cell.  M and K
  // are centrosymmetric (GLL nodes are symmetric), so each contraction splits
  // into an even part on s_b = u_b + u_{P-b} and an odd part on
  // d_b = u_b - u_{P-b}: (H+1)^2 + H^2 products instead of (P+1)^2 (H = P/2).
  constexpr int H = P / 2;
  using Acc = typename MacAcc<T>::type;  // multiply-accumulate chains (ds: unnormalised pairs)
  for (int it = tid; it < CELLS * NP; it += nth) {
    const int e = it / NP, ay = it - e * NP;
    const int ecy = e / E, ecx = e - ecy * E;
    const int gcx = ex0 + ecx, gcy = ey0 + ecy;
    if (gcx < 0 || gcx >= a.n || gcy < 0 || gcy >= a.n) continue;
    const C* row = su + (ecy * P + ay) * UT + ecx * P;
    C sv[H + 1], dv[H];
#pragma unroll
    for (int b = 0; b < H; ++b) {
      const C lo = row[b], hi = row[P - b];
      sv[b].x = lo.x + hi.x;
      sv[b].y = lo.y + hi.y;
      dv[b].x = lo.x - hi.x;
      dv[b].y = lo.y - hi.y;
    }
    sv[H] = row[H];
    C* o1 = s1 + (e * NP + ay) * NP;
    C* o2 = s2 + (e * NP + ay) * NP;
#pragma unroll
    for (int ax = 0; ax <= H; ++ax) {
      Acc pmr_{}, pmi_{}, pkr_{}, pki_{}, qmr_{}, qmi_{}, qkr_{}, qki_{};
#pragma unroll
      for (int b = 0; b <= H; ++b) {
        const T me = a.ME[ax * (H + 1) + b], ke = a.KE[ax * (H + 1) + b];
        mac(pmr_, me, sv[b].x);
        mac(pmi_, me, sv[b].y);
        mac(pkr_, ke, sv[b].x);
        mac(pki_, ke, sv[b].y);
      }
      const T pmr = mac_val(pmr_), pmi = mac_val(pmi_), pkr = mac_val(pkr_), pki = mac_val(pki_);
      if (ax < H) {
#pragma unroll
        for (int b = 0; b < H; ++b) {
          const T mo = a.MO[ax * H + b], ko = a.KO[ax * H + b];
          mac(qmr_, mo, dv[b].x);
          mac(qmi_, mo, dv[b].y);
          mac(qkr_, ko, dv[b].x);
          mac(qki_, ko, dv[b].y);
        }
        const T qmr = mac_val(qmr_), qmi = mac_val(qmi_), qkr = mac_val(qkr_), qki = mac_val(qki_);
        C t;
        t.x = pmr + qmr; t.y = pmi + qmi; o1[ax] = t;
        t.x = pmr - qmr; t.y = pmi - qmi; o1[P - ax] = t;
        t.x = pkr + qkr; t.y = pki + qki; o2[ax] = t;
        t.x = pkr - qkr; t.y = pki - qki; o2[P - ax] = t;
      } else {
        C t;
        t.x = pmr; t.y = pmi; o1[ax] = t;
        t.x = pkr; t.y = pki; o2[ax] = t;
      }
    }
  }
  __syncthreads();

  // phase 2: y-contractions, cell coefficient and absorbing boundary terms
  for (int it = tid; it < CELLS * NP; it += nth) {
    const int e = it / NP, ax = it - e * NP;
    const int ecy = e / E, ecx = e - ecy * E;
    const int gcx = ex0 + ecx, gcy = ey0 + ecy;
    if (gcx < 0 || gcx >= a.n || gcy < 0 || gcy >= a.n) continue;
    const T kk = skc[e], ee = sec[e];
    const T me_r = -kk * kk * a.h2, me_i = -(a.alpha * kk * kk + ee) * a.h2;
    C t1[NP], z[NP];
#pragma unroll
    for (int b = 0; b < NP; ++b) {
      t1[b] = s1[(e * NP + b) * NP + ax];
      const C t2 = s2[(e * NP + b) * NP + ax];
      const C mt = cmul(t1[b], me_r, me_i);
      z[b].x = t2.x + mt.x;
      z[b].y = t2.y + mt.y;
    }
    // y-contractions M z + K t1, split the same way
    C zs_[H + 1], zd_[H], ts_[H + 1], td_[H];
#pragma unroll
    for (int b = 0; b < H; ++b) {
      zs_[b].x = z[b].x + z[P - b].x;
      zs_[b].y = z[b].y + z[P - b].y;
      zd_[b].x = z[b].x - z[P - b].x;
      zd_[b].y = z[b].y - z[P - b].y;
      ts_[b].x = t1[b].x + t1[P - b].x;
      ts_[b].y = t1[b].y + t1[P - b].y;
      td_[b].x = t1[b].x - t1[P - b].x;
      td_[b].y = t1[b].y - t1[P - b].y;
    }
    zs_[H] = z[H];
    ts_[H] = t1[H];
    C yv[NP];
#pragma unroll
    for (int ay = 0; ay <= H; ++ay) {
      Acc pr_{}, pi_{}, qr_{}, qi_{};
#pragma unroll
      for (int b = 0; b <= H; ++b) {
        const T me = a.ME[ay * (H + 1) + b], ke = a.KE[ay * (H + 1) + b];
        mac_fma(pr_, me, zs_[b].x);
        mac_fma(pr_, ke, ts_[b].x);
        mac_fma(pi_, me, zs_[b].y);
        mac_fma(pi_, ke, ts_[b].y);
      }
      const T pr = mac_val(pr_), pi = mac_val(pi_);
      if (ay < H) {
#pragma unroll
        for (int b = 0; b < H; ++b) {
          const T mo = a.MO[ay * H + b], ko = a.KO[ay * H + b];
          mac_fma(qr_, mo, zd_[b].x);
          mac_fma(qr_, ko, td_[b].x);
          mac_fma(qi_, mo, zd_[b].y);
          mac_fma(qi_, ko, td_[b].y);
        }
        const T qr = mac_val(qr_), qi = mac_val(qi_);
        yv[ay].x = pr + qr;
        yv[ay].y = pi + qi;
        yv[P - ay].x = pr - qr;
        yv[P - ay].y = pi - qi;
      } else {
        yv[ay].x = pr;
        yv[ay].y = pi;
      }
    }
    // -i k h M on absorbing sides: rho * (x + i y) = k h y - i k h x
    const T kh = kk * a.h;
    if (gcy == 0 && (a.robin & 4)) { yv[0].x += kh * t1[0].y; yv[0].y -= kh * t1[0].x; }
    if (gcy == a.n - 1 && (a.robin & 8)) { yv[P].x += kh * t1[P].y; yv[P].y -= kh * t1[P].x; }
    if ((ax == 0 && gcx == 0 && (a.robin & 1)) || (ax == P && gcx == a.n - 1 && (a.robin & 2))) {
      const C* col = su + (ecy * P) * UT + ecx * P + ax;
#pragma unroll
      for (int ay = 0; ay < NP; ++ay) {
        T sr = 0, si = 0;
#pragma unroll
        for (int b = 0; b < NP; ++b) {
          const T mm = a.M[ay * NP + b];
          sr += mm * col[b * UT].x;
          si += mm * col[b * UT].y;
        }
        yv[ay].x += kh * si;
        yv[ay].y -= kh * sr;
      }
    }
#pragma unroll
    for (int ay = 0; ay < NP; ++ay) s2[(e * NP + ay) * NP + ax] = yv[ay];
  }
  __syncthreads();

  // phase 3: owned nodes sum their cells in a fixed order
  // output and right-hand side addressed from their bases: the double-single
  // variant's output elements are narrower than C (see NodeIO<ds>)
  for (int i = tid; i < wx * wy; i += nth) {
    const int ly = i / wx, lx = i - ly * wx;
    const int ux = lx + P, uy = ly + P;
    int exs[2], axs[2], eys[2], ays[2];
    int nxc = 0, nyc = 0;
    if (ux % P == 0) {
      exs[nxc] = ux / P - 1; axs[nxc++] = P;
      exs[nxc] = ux / P;     axs[nxc++] = 0;
    } else {
      exs[nxc] = ux / P; axs[nxc++] = ux % P;
    }
    if (uy % P == 0) {
      eys[nyc] = uy / P - 1; ays[nyc++] = P;
      eys[nyc] = uy / P;     ays[nyc++] = 0;
    } else {
      eys[nyc] = uy / P; ays[nyc++] = uy % P;
    }
    T ar = 0, ai = 0;
    for (int jy = 0; jy < nyc; ++jy) {
      const int ey = eys[jy], gcy = ey0 + ey;
      if (ey >= E || gcy < 0 || gcy >= a.n) continue;
      for (int jx = 0; jx < nxc; ++jx) {
        const int ex = exs[jx], gcx = ex0 + ex;
        if (ex >= E || gcx < 0 || gcx >= a.n) continue;
        const C v = s2[((ey * E + ex) * NP + ays[jy]) * NP + axs[jx]];
        ar += v.x;
        ai += v.y;
      }
    }
    const size_t g = (size_t)(cy0 * P + ly) * a.m + (cx0 * P + lx);
    const int gx = cx0 * P + lx, gy = cy0 * P + ly;
    C uo = su[(ly + P) * UT + lx + P];
    if (a.dirichlet && (((a.dirichlet & 1) && gx == 0) || ((a.dirichlet & 2) && gx == a.m - 1) ||
                        ((a.dirichlet & 4) && gy == 0) || ((a.dirichlet & 8) && gy == a.m - 1))) {
      // identity row on Gamma_0: (A u)_j = u_j, with the operand's own value
      if constexpr (std::is_same<T, ds>::value) {
        uo = NodeIO<T>::ld(u, g);
      } else {
        uo = a.src == 1 ? combine_at(a, gx, gy) : a.src == 2 ? prolong_at(a, gx, gy) : NodeIO<T>::ld(u, g);
      }
      ar = uo.x;
      ai = uo.y;
    }
    if constexpr (!std::is_same<T, ds>::value) {
      if (a.src != 0) a.uout[roff + g] = uo;
    }
    C out;
    if (a.f) {
      out.x = sf[i].x - ar;
      out.y = sf[i].y - ai;
    } else {
      out.x = ar;
      out.y = ai;
    }
    if constexpr (std::is_same<T, ds>::value) {
      if (a.out64) {  // FP64 output (the FGMRES product A z of the mixed form)
        reinterpret_cast<double2*>(a.y)[roff + g] =
            make_double2(f2d_bits(out.x.h) + f2d_bits(out.x.l), f2d_bits(out.y.h) + f2d_bits(out.y.l));
        continue;
      }
    }
    NodeIO<T>::st(a.y, roff + g, out);
  }
}

template <int P, int TC, typename T>
static cudaError_t launch_fine_p(const FineArgs<T>& a, int nrhs, cudaStream_t s) {
  using C = typename Cx<T>::t;
  constexpr int NP = P + 1, E = TC + 1, UT = E * P + 1;
  const size_t smem = sizeof(C) * (size_t)(UT * UT + 2 * E * E * NP * NP + (TC * P + 1) * (TC * P + 1)) +
                      sizeof(T) * 2 * E * E;
  // set on every launch (a cheap host call): the attribute is per device, and
  // any device of the process may run this instantiation
  cudaError_t e = cudaFuncSetAttribute(k_fine_apply<P, TC, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles = (a.n + TC - 1) / TC;
  dim3 grid(tiles, tiles, nrhs);
  return launch_pdl(k_fine_apply<P, TC, T>, grid, dim3(TC >= 8 ? 256 : 128), smem, s, 0, a);
}

template <typename T>
cudaError_t launch_fine_apply(const FineArgs<T>& a, int nrhs, cudaStream_t s) {
  // two tile shapes per order: the larger recomputes fewer halo cells, the
  // smaller spreads a small mesh over more SMs (chosen by the set-up autotuner)
  const bool small = (a.tc != 0);
  switch (a.p) {
    case 2: return small ? launch_fine_p<2, 8, T>(a, nrhs, s) : launch_fine_p<2, 16, T>(a, nrhs, s);
    case 4: return small ? launch_fine_p<4, 4, T>(a, nrhs, s) : launch_fine_p<4, 8, T>(a, nrhs, s);
    case 6: return small ? launch_fine_p<6, 3, T>(a, nrhs, s) : launch_fine_p<6, 5, T>(a, nrhs, s);
    case 8: return small ? launch_fine_p<8, 2, T>(a, nrhs, s) : launch_fine_p<8, 4, T>(a, nrhs, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_fine_apply<double>(const FineArgs<double>&, int, cudaStream_t);
template cudaError_t launch_fine_apply<float>(const FineArgs<float>&, int, cudaStream_t);
template cudaError_t launch_fine_apply<ds>(const FineArgs<ds>&, int, cudaStream_t);

}  // namespace th
