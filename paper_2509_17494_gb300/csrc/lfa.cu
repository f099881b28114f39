// Local Fourier analysis of the finite-element two-grid method on the GPU
// (Section 6, Eq. symbol_sum): for constant k and eps on the periodic plane,
// the Bloch symbols of A, A_s, the QSFEM coarse operator A_c and the transfers
// are sums over the neighbour cells beta of exp(i theta . beta) P_{0,beta};
// M(theta) = S^{n_s} K S^{n_s}, S = I - A_s^{-1} A (exact shifted smoother),
// K = I - omega_c I_P A_c^{-1} I_R A, and the method's asymptotic rate is
// sup_theta rho(M(theta)).  A_c is the QSFEM operator ('opt') or the Galerkin
// operator I_R A_{alpha_c} I_P of standard p-type coarsening ('gal', Fig. 3 (a)).
//
// Host: the blocks P_{0,beta} from a dense assembly on a periodic torus of
// 3 x 3 cells (every operator reaches one cell at most, so no block aliases),
// per parameter point.  Device (K17 k_lfa): one CTA per (parameter point,
// theta): the symbols, Gaussian elimination with partial pivoting for
// A_s^{-1} A and A_c^{-1} I_R A, the products, and rho(M) by Gelfand's formula
// rho = lim ||M^(2^J)||^(1/2^J), evaluated by J normalised squarings:
// log rho ~ sum_j 2^-j log s_j, s_j the Frobenius norm before the j-th
// normalisation.  For J = 40 the limit error is below (log kappa + n log 2^J) / 2^J,
// about 1e-10 relative for these matrices.
#include <cmath>
#include <complex>
#include <vector>

#include "th_internal.h"

namespace th {

namespace {

constexpr int kLfaJ = 40;

struct LfaDims {
  int p, q, n, nc;  // fine / coarse unit-cell dofs n = p^2, nc = q^2
};

// Dense periodic assembly on a 3 x 3-cell torus with h = 1 (the 2-D forms
// depend on k and eps only through k h and eps h^2), then the blocks.
void lfa_blocks(const Ref1D& ref, const LfaDims& d, double kh, double eps_k2, double alpha_s, int gal,
                double alpha_c, std::vector<cplx>& A, std::vector<cplx>& As, std::vector<cplx>& Ac,
                std::vector<double>* IP, std::vector<double>* IR) {
  const int p = d.p, q = d.q, np = p + 1, mf = 3 * p, mcn = 3 * q;
  const int Nf = mf * mf, Ncn = mcn * mcn;
  std::vector<cplx> Af((size_t)Nf * Nf, 0.0), Asf((size_t)Nf * Nf, 0.0), Acf((size_t)Ncn * Ncn, 0.0);
  const double k = kh, eps = eps_k2 * kh * kh;
  const cplx cA(k * k, eps), cS(k * k, alpha_s * k * k + eps);
  for (int cy = 0; cy < 3; ++cy)
    for (int cx = 0; cx < 3; ++cx)
      for (int ay = 0; ay < np; ++ay)
        for (int ax = 0; ax < np; ++ax)
          for (int by = 0; by < np; ++by)
            for (int bx = 0; bx < np; ++bx) {
              const int r = ((cy * p + ay) % mf) * mf + (cx * p + ax) % mf;
              const int c = ((cy * p + by) % mf) * mf + (cx * p + bx) % mf;
              const double my = ref.M[ay * np + by], mx = ref.M[ax * np + bx];
              const double ky = ref.K[ay * np + by], kx = ref.K[ax * np + bx];
              const double st = kx * my + mx * ky, ms = mx * my;
              Af[(size_t)r * Nf + c] += st - cA * ms;
              Asf[(size_t)r * Nf + c] += st - cS * ms;
            }
  // prolongation on the torus: fine node i (1-D) = cell e, local a; coarse J = e q + b
  std::vector<double> P1((size_t)mf * mcn, 0.0);
  for (int e = 0; e < 3; ++e)
    for (int a = 0; a <= p; ++a)
      for (int b = 0; b <= q; ++b) P1[(size_t)((e * p + a) % mf) * mcn + (e * q + b) % mcn] = ref.Pw[a * (q + 1) + b];
  if (!gal) {
    // QSFEM coarse cells (spacing h / q): pair weights by the number of differing coordinates
    const double hc = 1.0 / q;
    cplx dq[3];
    qsfem_cell(k, eps, hc, dq);
    for (int cy = 0; cy < mcn; ++cy)
      for (int cx = 0; cx < mcn; ++cx)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            const int ay = cy + (a >> 1), ax = cx + (a & 1), by = cy + (b >> 1), bx = cx + (b & 1);
            const int nd = (ax != bx) + (ay != by);
            const int r = (ay % mcn) * mcn + ax % mcn, c = (by % mcn) * mcn + bx % mcn;
            Acf[(size_t)r * Ncn + c] += dq[nd];
          }
  } else {
    // Galerkin: A_c = I_P^T A_{alpha_c} I_P on the torus, I_P = P1 (x) P1
    const cplx cG(k * k, alpha_c * k * k + eps);
    std::vector<cplx> Ag((size_t)Nf * Nf, 0.0);
    for (int cy = 0; cy < 3; ++cy)
      for (int cx = 0; cx < 3; ++cx)
        for (int ay = 0; ay < np; ++ay)
          for (int ax = 0; ax < np; ++ax)
            for (int by = 0; by < np; ++by)
              for (int bx = 0; bx < np; ++bx) {
                const int r = ((cy * p + ay) % mf) * mf + (cx * p + ax) % mf;
                const int c = ((cy * p + by) % mf) * mf + (cx * p + bx) % mf;
                const double my = ref.M[ay * np + by], mx = ref.M[ax * np + bx];
                const double ky = ref.K[ay * np + by], kx = ref.K[ax * np + bx];
                Ag[(size_t)r * Nf + c] += (kx * my + mx * ky) - cG * (mx * my);
              }
    // T = Ag I_P (Nf x Ncn), then Acf = I_P^T T
    std::vector<cplx> T((size_t)Nf * Ncn, 0.0);
    for (int r = 0; r < Nf; ++r)
      for (int c = 0; c < Nf; ++c) {
        const cplx v = Ag[(size_t)r * Nf + c];
        if (v == 0.0) continue;
        const int fy = c / mf, fx = c % mf;
        for (int J = 0; J < Ncn; ++J) {
          const double w = P1[(size_t)fy * mcn + J / mcn] * P1[(size_t)fx * mcn + J % mcn];
          if (w != 0.0) T[(size_t)r * Ncn + J] += v * w;
        }
      }
    for (int r = 0; r < Nf; ++r) {
      const int fy = r / mf, fx = r % mf;
      for (int I = 0; I < Ncn; ++I) {
        const double w = P1[(size_t)fy * mcn + I / mcn] * P1[(size_t)fx * mcn + I % mcn];
        if (w == 0.0) continue;
        for (int J = 0; J < Ncn; ++J) Acf[(size_t)I * Ncn + J] += w * T[(size_t)r * Ncn + J];
      }
    }
  }
  // blocks: rows of the unit cell of cell (0, 0), columns of the unit cell of cell beta
  auto fine_idx = [&](int by, int bx, int a) {
    const int ay = a / p, ax = a % p;
    return (((by + 3) % 3) * p + ay) * mf + ((bx + 3) % 3) * p + ax;
  };
  auto coarse_idx = [&](int by, int bx, int a) {
    const int ay = a / q, ax = a % q;
    return (((by + 3) % 3) * q + ay) * mcn + ((bx + 3) % 3) * q + ax;
  };
  A.assign((size_t)9 * d.n * d.n, 0.0);
  As.assign((size_t)9 * d.n * d.n, 0.0);
  Ac.assign((size_t)9 * d.nc * d.nc, 0.0);
  if (IP) IP->assign((size_t)9 * d.n * d.nc, 0.0);
  if (IR) IR->assign((size_t)9 * d.nc * d.n, 0.0);
  for (int bi = 0; bi < 9; ++bi) {
    const int by = bi / 3 - 1, bx = bi % 3 - 1;
    for (int r = 0; r < d.n; ++r) {
      const int gr = fine_idx(0, 0, r);
      for (int c = 0; c < d.n; ++c) {
        const int gc = fine_idx(by, bx, c);
        A[((size_t)bi * d.n + r) * d.n + c] = Af[(size_t)gr * Nf + gc];
        As[((size_t)bi * d.n + r) * d.n + c] = Asf[(size_t)gr * Nf + gc];
      }
      if (IP)
        for (int c = 0; c < d.nc; ++c) {
          const int gc = coarse_idx(by, bx, c);
          const int fy = gr / mf, fx = gr % mf, Jy = gc / mcn, Jx = gc % mcn;
          (*IP)[((size_t)bi * d.n + r) * d.nc + c] = P1[(size_t)fy * mcn + Jy] * P1[(size_t)fx * mcn + Jx];
        }
    }
    for (int r = 0; r < d.nc; ++r) {
      const int gr = coarse_idx(0, 0, r);
      for (int c = 0; c < d.nc; ++c) Ac[((size_t)bi * d.nc + r) * d.nc + c] = Acf[(size_t)gr * Ncn + coarse_idx(by, bx, c)];
      if (IR)
        for (int c = 0; c < d.n; ++c) {
          const int gc = fine_idx(by, bx, c);
          const int Jy = gr / mcn, Jx = gr % mcn, fy = gc / mf, fx = gc % mf;
          (*IR)[((size_t)bi * d.nc + r) * d.n + c] = P1[(size_t)fy * mcn + Jy] * P1[(size_t)fx * mcn + Jx];
        }
    }
  }
}

struct LfaArgs {
  const double2* A;    // [param][9][n][n]
  const double2* As;   // [param][9][n][n]
  const double2* Ac;   // [param][9][nc][nc]
  const double* IP;    // [9][n][nc]
  const double* IR;    // [9][nc][n]
  const double* omega; // [param]
  double* rho;         // [param][npts^2]
  int n, nc, npts, n_s, nparam;
};

__device__ __forceinline__ double2 cmulz(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// C[n x m] = sum_beta e^{i theta.beta} B_beta (complex blocks)
__device__ void lfa_symbol(const double2* B, int n, int m, double ty, double tx, double2* C) {
  for (int i = threadIdx.x; i < n * m; i += blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int bi = 0; bi < 9; ++bi) {
      double sn, cs;
      sincos(ty * (bi / 3 - 1) + tx * (bi % 3 - 1), &sn, &cs);
      const double2 v = B[(size_t)bi * n * m + i];
      s.x += cs * v.x - sn * v.y;
      s.y += cs * v.y + sn * v.x;
    }
    C[i] = s;
  }
}
__device__ void lfa_symbol_real(const double* B, int n, int m, double ty, double tx, double2* C) {
  for (int i = threadIdx.x; i < n * m; i += blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int bi = 0; bi < 9; ++bi) {
      double sn, cs;
      sincos(ty * (bi / 3 - 1) + tx * (bi % 3 - 1), &sn, &cs);
      const double v = B[(size_t)bi * n * m + i];
      s.x += cs * v;
      s.y += sn * v;
    }
    C[i] = s;
  }
}

// X <- A^{-1} X (A n x n, X n x m; A is overwritten): Gauss-Jordan elimination
// with partial pivoting on [A | X], the rows left unscaled until the end
__device__ void lfa_solve(double2* Am, int n, double2* X, int m, int* piv) {
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int pr = k;
      double best = hypot(Am[k * n + k].x, Am[k * n + k].y);
      for (int r = k + 1; r < n; ++r) {
        const double v = hypot(Am[r * n + k].x, Am[r * n + k].y);
        if (v > best) { best = v; pr = r; }
      }
      *piv = pr;
    }
    __syncthreads();
    const int pr = *piv;
    if (pr != k) {
      for (int c = threadIdx.x; c < n + m; c += blockDim.x) {
        double2* a = c < n ? &Am[k * n + c] : &X[k * m + c - n];
        double2* b = c < n ? &Am[pr * n + c] : &X[pr * m + c - n];
        const double2 t = *a;
        *a = *b;
        *b = t;
      }
    }
    __syncthreads();
    const double2 pv = Am[k * n + k];
    const double den = pv.x * pv.x + pv.y * pv.y;
    const double2 inv = make_double2(pv.x / den, -pv.y / den);
    // eliminate column k from every other row (Gauss-Jordan), rows r != k
    for (int idx = threadIdx.x; idx < (n - 1) * (n - k - 1 + m); idx += blockDim.x) {
      const int w = n - k - 1 + m;
      int r = idx / w;
      if (r >= k) ++r;
      const int cc = idx % w;
      const double2 f = cmulz(Am[r * n + k], inv);
      if (cc < n - k - 1) {
        const int c = k + 1 + cc;
        const double2 t = cmulz(f, Am[k * n + c]);
        Am[r * n + c].x -= t.x;
        Am[r * n + c].y -= t.y;
      } else {
        const int c = cc - (n - k - 1);
        const double2 t = cmulz(f, X[k * m + c]);
        X[r * m + c].x -= t.x;
        X[r * m + c].y -= t.y;
      }
    }
    __syncthreads();
    // column k of the other rows is now zero in exact arithmetic (it is not stored)
  }
  // A is diagonal: X <- D^{-1} X
  for (int i = threadIdx.x; i < n * m; i += blockDim.x) {
    const double2 pv = Am[(i / m) * n + i / m];
    const double den = pv.x * pv.x + pv.y * pv.y;
    X[i] = cmulz(X[i], make_double2(pv.x / den, -pv.y / den));
  }
  __syncthreads();
}

// C = A B (n x l, l x m), complex, C distinct from A and B
__device__ void lfa_mm(const double2* A, const double2* B, double2* C, int n, int l, int m) {
  for (int i = threadIdx.x; i < n * m; i += blockDim.x) {
    const int r = i / m, c = i % m;
    double2 s = make_double2(0.0, 0.0);
    for (int t = 0; t < l; ++t) {
      const double2 a = A[r * l + t], b = B[t * m + c];
      s.x = fma(a.x, b.x, s.x);
      s.x = fma(-a.y, b.y, s.x);
      s.y = fma(a.x, b.y, s.y);
      s.y = fma(a.y, b.x, s.y);
    }
    C[i] = s;
  }
  __syncthreads();
}

__device__ double lfa_fro(const double2* X, int len, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) s += X[i].x * X[i].x + X[i].y * X[i].y;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return sqrt(t);
}

__global__ void __launch_bounds__(256) k_lfa(const LfaArgs a) {
  extern __shared__ __align__(16) unsigned char lfa_sm[];
  const int n = a.n, nc = a.nc, nn = n * n;
  double2* S = reinterpret_cast<double2*>(lfa_sm);  // n x n
  double2* M = S + nn;                               // n x n
  double2* T1 = M + nn;                              // n x n
  double2* T2 = T1 + nn;                             // n x n
  double2* Q = T2 + nn;                              // nc x n
  double2* Cc = Q + nc * n;                          // nc x nc
  double2* Pm = Cc + nc * nc;                        // n x nc
  double2* Rm = Pm + n * nc;                         // nc x n
  double* red = reinterpret_cast<double*>(Rm + nc * n);  // [32]
  __shared__ int piv;
  const int param = blockIdx.y, tj = blockIdx.x;
  const int iy = tj / a.npts, ix = tj % a.npts;
  const double ty = -M_PI + 2.0 * M_PI * iy / a.npts, tx = -M_PI + 2.0 * M_PI * ix / a.npts;
  const double2* Ab = a.A + (size_t)param * 9 * nn;
  // S = I - A_s^{-1} A
  lfa_symbol(a.As + (size_t)param * 9 * nn, n, n, ty, tx, T1);
  lfa_symbol(Ab, n, n, ty, tx, S);
  __syncthreads();
  lfa_solve(T1, n, S, n, &piv);  // S = A_s^{-1} A
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int r = i / n, c = i % n;
    S[i] = make_double2((r == c ? 1.0 : 0.0) - S[i].x, -S[i].y);
  }
  // K = I - omega I_P A_c^{-1} I_R A
  lfa_symbol(Ab, n, n, ty, tx, T2);
  lfa_symbol(a.Ac + (size_t)param * 9 * nc * nc, nc, nc, ty, tx, Cc);
  lfa_symbol_real(a.IP, n, nc, ty, tx, Pm);
  lfa_symbol_real(a.IR, nc, n, ty, tx, Rm);
  __syncthreads();
  lfa_mm(Rm, T2, Q, nc, n, n);  // Q = I_R A
  lfa_solve(Cc, nc, Q, n, &piv);  // Q = A_c^{-1} I_R A
  lfa_mm(Pm, Q, T1, n, nc, n);  // T1 = I_P A_c^{-1} I_R A
  const double om = a.omega[param];
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int r = i / n, c = i % n;
    T1[i] = make_double2((r == c ? 1.0 : 0.0) - om * T1[i].x, -om * T1[i].y);  // K
  }
  __syncthreads();
  // M = S^{n_s} K S^{n_s}
  for (int i = threadIdx.x; i < nn; i += blockDim.x) M[i] = T1[i];
  __syncthreads();
  for (int s = 0; s < a.n_s; ++s) {
    lfa_mm(M, S, T2, n, n, n);
    lfa_mm(S, T2, M, n, n, n);
  }
  // Gelfand: J normalised squarings
  double lg = 0.0, w = 1.0;
  double nrm = lfa_fro(M, nn, red);
  for (int j = 0; j <= kLfaJ; ++j) {
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      lg = nrm > 0.0 ? INFINITY : -INFINITY;
      break;
    }
    lg += w * log(nrm);
    if (j == kLfaJ) break;
    const double inv = 1.0 / nrm;
    for (int i = threadIdx.x; i < nn; i += blockDim.x) M[i] = make_double2(M[i].x * inv, M[i].y * inv);
    __syncthreads();
    lfa_mm(M, M, T2, n, n, n);
    for (int i = threadIdx.x; i < nn; i += blockDim.x) M[i] = T2[i];
    __syncthreads();
    nrm = lfa_fro(M, nn, red);
    w *= 0.5;
  }
  if (threadIdx.x == 0) a.rho[(size_t)param * a.npts * a.npts + tj] = exp(lg);
}

}  // namespace

}  // namespace th

th_status th_lfa_rho(int p, int n_s, int npts, int coarse_kind, double alpha_c, const double* params, int nparam,
                     double* rho_max, double* rho_theta, void* stream) {
  using th::cplx;
  if (!params || !rho_max || nparam < 1 || npts < 1 || npts > 4096 || n_s < 0 || n_s > 8) return TH_ERR_ARG;
  if (p != 2 && p != 4 && p != 6) return TH_ERR_UNSUPPORTED;
  if ((coarse_kind != TH_CK_QSFEM && coarse_kind != TH_CK_GALERKIN) || !std::isfinite(alpha_c) || alpha_c < 0.0)
    return TH_ERR_ARG;
  for (int i = 0; i < 4 * nparam; ++i)
    if (!std::isfinite(params[i])) return TH_ERR_ARG;
  for (int i = 0; i < nparam; ++i)
    if (!(params[4 * i] > 0.0) || params[4 * i + 1] < 0.0 || params[4 * i + 2] < 0.0) return TH_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  th::LfaDims d{p, p / 2, p * p, (p / 2) * (p / 2)};
  const th::Ref1D ref = th::reference_1d(p);
  std::vector<double2> hA, hAs, hAc;
  std::vector<double> IP, IR, om(nparam);
  for (int i = 0; i < nparam; ++i) {
    std::vector<cplx> A, As, Ac;
    th::lfa_blocks(ref, d, params[4 * i], params[4 * i + 1], params[4 * i + 2], coarse_kind == TH_CK_GALERKIN,
                   alpha_c, A, As, Ac, i == 0 ? &IP : nullptr, i == 0 ? &IR : nullptr);
    for (const cplx& v : A) hA.push_back(make_double2(v.real(), v.imag()));
    for (const cplx& v : As) hAs.push_back(make_double2(v.real(), v.imag()));
    for (const cplx& v : Ac) hAc.push_back(make_double2(v.real(), v.imag()));
    om[i] = params[4 * i + 3];
  }
  const size_t ntheta = (size_t)npts * npts;
  std::vector<double> hr(ntheta * nparam);
  // device buffers of this call (the analysis is not on the two-grid path)
  double2 *dA = nullptr, *dAs = nullptr, *dAc = nullptr;
  double *dIP = nullptr, *dIR = nullptr, *dom = nullptr, *drho = nullptr;
  th_status st = TH_OK;
  auto al = [&](void** ptr, size_t bytes) {
    if (st == TH_OK && cudaMalloc(ptr, bytes) != cudaSuccess) st = TH_ERR_NOMEM;
  };
  al((void**)&dA, hA.size() * 16);
  al((void**)&dAs, hAs.size() * 16);
  al((void**)&dAc, hAc.size() * 16);
  al((void**)&dIP, IP.size() * 8);
  al((void**)&dIR, IR.size() * 8);
  al((void**)&dom, om.size() * 8);
  al((void**)&drho, hr.size() * 8);
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (st == TH_OK && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) st = TH_ERR_CUDA;
  };
  cp(dA, hA.data(), hA.size() * 16);
  cp(dAs, hAs.data(), hAs.size() * 16);
  cp(dAc, hAc.data(), hAc.size() * 16);
  cp(dIP, IP.data(), IP.size() * 8);
  cp(dIR, IR.data(), IR.size() * 8);
  cp(dom, om.data(), om.size() * 8);
  if (st == TH_OK) {
    th::LfaArgs a{dA, dAs, dAc, dIP, dIR, dom, drho, d.n, d.nc, npts, n_s, nparam};
    const size_t smem = (size_t)16 * (4 * d.n * d.n + 3 * d.nc * d.n + d.nc * d.nc) + 32 * 8;
    cudaError_t e = cudaFuncSetAttribute(th::k_lfa, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      th::k_lfa<<<dim3((unsigned)ntheta, nparam), 256, smem, s>>>(a);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = TH_ERR_CUDA;
  }
  if (st == TH_OK && cudaMemcpyAsync(hr.data(), drho, hr.size() * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    st = TH_ERR_CUDA;
  if (st == TH_OK && cudaStreamSynchronize(s) != cudaSuccess) st = TH_ERR_CUDA;
  cudaFree(dA);
  cudaFree(dAs);
  cudaFree(dAc);
  cudaFree(dIP);
  cudaFree(dIR);
  cudaFree(dom);
  cudaFree(drho);
  if (st != TH_OK) return st;
  for (int i = 0; i < nparam; ++i) {
    double mx = 0.0;
    for (size_t t = 0; t < ntheta; ++t) mx = std::max(mx, hr[(size_t)i * ntheta + t]);
    rho_max[i] = mx;
  }
  if (rho_theta) std::copy(hr.begin(), hr.end(), rho_theta);
  return TH_OK;
}
