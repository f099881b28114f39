// K18: the dispersion error D_P of a compact 2-D stencil (Section 3.2).
//
// A symmetric 3 x 3 stencil with centre P0, edge P1 and corner P2 has the
// symbol sigma(z) = P0 + 2 P1 (cos z1 + cos z2) + 4 P2 cos z1 cos z2 (z = h xi,
// Eq. symbol_sigma_P); its propagating waves are the zero set Z_P, and
//   D_P = max over t of min over xi in Z_P of |k (cos t, sin t) - xi| ,
// here divided by k (eta = k h, all lengths in units of 1/h).  One thread per
// (stencil, direction t): the zero set along a ray of polar angle s is the
// first sign change of sigma on a grid of the ray, refined by bisection to
// full precision; the distance |eta e_t - r(s) e_s|^2 = (r - eta)^2 +
// 4 eta r sin^2((s - t)/2) is minimised over s on a grid around t, then by
// golden-section search in the bracketing cells.  FP64 throughout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "th.h"
#include "th_internal.h"

namespace th {
namespace {

struct DispArgs {
  const double* P;  // [n][4]: P0, P1, P2, eta
  double* d;        // [n][nt]
  int n, nt;
};

__device__ double disp_symbol(const double* P, double z1, double z2) {
  const double c1 = cos(z1), c2 = cos(z2);
  return P[0] + 2.0 * P[1] * (c1 + c2) + 4.0 * P[2] * c1 * c2;
}

// smallest r > 0 with sigma(r e_s) = 0; negative if the ray has no zero
__device__ double disp_radius(const double* P, double s) {
  const double eta = P[3], cs = cos(s), sn = sin(s);
  constexpr int NR = 512;
  const double r0 = 1e-3 * eta, r1 = 3.0 * fmax(eta, 0.5);
  double a = r0, fa = disp_symbol(P, r0 * cs, r0 * sn);
  for (int i = 1; i <= NR; ++i) {
    const double b = r0 + (r1 - r0) * i / NR;
    const double fb = disp_symbol(P, b * cs, b * sn);
    if ((fa < 0.0) != (fb < 0.0)) {
      double lo = a, hi = b, flo = fa;
      for (int it = 0; it < 80 && hi - lo > 1e-16 * hi; ++it) {
        const double m = 0.5 * (lo + hi);
        const double fm = disp_symbol(P, m * cs, m * sn);
        if ((flo < 0.0) != (fm < 0.0)) {
          hi = m;
        } else {
          lo = m;
          flo = fm;
        }
      }
      return 0.5 * (lo + hi);
    }
    a = b;
    fa = fb;
  }
  return -1.0;
}

__device__ double disp_d2(const double* P, double s, double t) {
  const double eta = P[3];
  const double r = disp_radius(P, s);
  if (r < 0.0) return 1e300;
  const double h = sin(0.5 * (s - t));
  return (r - eta) * (r - eta) + 4.0 * eta * r * h * h;
}

__global__ void __launch_bounds__(128) k_dispersion(const DispArgs a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= a.nt || i >= a.n) return;
  const double* P = a.P + (size_t)i * 4;
  const double pi = 3.141592653589793238462643383279502884;
  const double t = -pi + 2.0 * pi * j / a.nt;
  constexpr int NS = 61;
  constexpr double W = 0.3;
  double best = 1e300;
  int ib = 0;
  for (int q = 0; q < NS; ++q) {
    const double s = t - W + 2.0 * W * q / (NS - 1);
    const double v = disp_d2(P, s, t);
    if (v < best) {
      best = v;
      ib = q;
    }
  }
  double lo = t - W + 2.0 * W * max(ib - 1, 0) / (NS - 1);
  double hi = t - W + 2.0 * W * min(ib + 1, NS - 1) / (NS - 1);
  const double g = 0.6180339887498948482;
  double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
  double f1 = disp_d2(P, x1, t), f2 = disp_d2(P, x2, t);
  for (int it = 0; it < 90 && hi - lo > 1e-13; ++it) {
    if (f1 < f2) {
      hi = x2;
      x2 = x1;
      f2 = f1;
      x1 = hi - g * (hi - lo);
      f1 = disp_d2(P, x1, t);
    } else {
      lo = x1;
      x1 = x2;
      f1 = f2;
      x2 = lo + g * (hi - lo);
      f2 = disp_d2(P, x2, t);
    }
  }
  best = fmin(best, fmin(f1, f2));
  a.d[(size_t)i * a.nt + j] = sqrt(fmax(best, 0.0)) / P[3];
}

}  // namespace
}  // namespace th

extern "C" th_status th_dispersion(int kind, const double* eta, int n, int nt, double* d_max, double* d_theta,
                                   void* stream) {
  if (!eta || !d_max || n < 1 || nt < 1 || nt > (1 << 20)) return TH_ERR_ARG;
  if (kind != TH_DISP_QSFEM && kind != TH_DISP_Q1 && kind != TH_DISP_FD5) return TH_ERR_ARG;
  std::vector<double> hp((size_t)n * 4);
  for (int i = 0; i < n; ++i) {
    const double e = eta[i];
    if (!std::isfinite(e) || e <= 0.0 || e > 2.0) return TH_ERR_ARG;
    double* P = &hp[(size_t)i * 4];
    if (kind == TH_DISP_QSFEM) {
      // assembled stencil from the per-cell weights N P0/4, N P1/2, N P2 (eps = 0, h = 1)
      th::cplx c[3];
      th::qsfem_cell(e, 0.0, 1.0, c);
      P[0] = 4.0 * c[0].real();
      P[1] = 2.0 * c[1].real();
      P[2] = c[2].real();
    } else if (kind == TH_DISP_Q1) {
      // Q1 stiffness minus eta^2 times the Q1 mass (Section 3.3)
      P[0] = 8.0 / 3.0 - 16.0 * e * e / 36.0;
      P[1] = -1.0 / 3.0 - 4.0 * e * e / 36.0;
      P[2] = -1.0 / 3.0 - e * e / 36.0;
    } else {
      P[0] = 4.0 - e * e;
      P[1] = -1.0;
      P[2] = 0.0;
    }
    P[3] = e;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<double> hd((size_t)n * nt);
  double *dP = nullptr, *dd = nullptr;
  th_status st = TH_OK;
  if (cudaMalloc((void**)&dP, hp.size() * 8) != cudaSuccess) st = TH_ERR_NOMEM;
  if (st == TH_OK && cudaMalloc((void**)&dd, hd.size() * 8) != cudaSuccess) st = TH_ERR_NOMEM;
  if (st == TH_OK && cudaMemcpyAsync(dP, hp.data(), hp.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
    st = TH_ERR_CUDA;
  if (st == TH_OK) {
    th::DispArgs a{dP, dd, n, nt};
    th::k_dispersion<<<dim3((unsigned)((nt + 127) / 128), (unsigned)n), 128, 0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) st = TH_ERR_CUDA;
  }
  if (st == TH_OK && cudaMemcpyAsync(hd.data(), dd, hd.size() * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    st = TH_ERR_CUDA;
  if (st == TH_OK && cudaStreamSynchronize(s) != cudaSuccess) st = TH_ERR_CUDA;
  cudaFree(dP);
  cudaFree(dd);
  if (st != TH_OK) return st;
  for (int i = 0; i < n; ++i) {
    double mx = 0.0;
    for (int j = 0; j < nt; ++j) mx = std::max(mx, hd[(size_t)i * nt + j]);
    d_max[i] = mx;
  }
  if (d_theta) std::copy(hd.begin(), hd.end(), d_theta);
  return TH_OK;
}
