// Host-side FP64 set-up of the two-grid Helmholtz library.
//
//  * 1-D reference element (Section 3.1): GLL nodes by Newton iteration on
//    P_p', exact mass/stiffness with a (p+2)-point Gauss-Legendre rule, the
//    derivatives through the barycentric differentiation matrix.
//  * Partition and overlapping subdomains (Section 4.1, Section 4.5).
//  * Subdomain matrices A_s^(i) (shifted volume coefficient, unshifted -i k
//    on internal boundaries, inherited conditions elsewhere) and their
//    inverse rows on the dofs of U^(i), scaled by 1/L_j (Eq. RAS_like_update),
//    by a banded LU with partial pivoting.
//  * QSFEM coarse cell coefficients (Eq. P_QSFEM, Eq. scaling_factor_QSFEM,
//    Eq. element_wise_qsfem) and the block-tridiagonal factorisation of A_q
//    by coarse grid rows.
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <thread>

#include "th_internal.h"

namespace th {

// ------------------------------------------------------------------ threads
void parallel_for(int n, const std::function<void(int)>& f) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = (int)std::max(1u, std::min(hw == 0 ? 4u : hw, 64u));
  nt = std::min(nt, n);
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int> next(0);
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&]() {
      for (;;) {
        int i = next.fetch_add(1);
        if (i >= n) break;
        f(i);
      }
    });
  for (auto& th : pool) th.join();
}

// ------------------------------------------------------------- 1-D element
static void legendre_pd(int n, double x, double& P, double& dP) {
  // P_n(x) and P_n'(x) by the three-term recurrence (|x| < 1 for dP)
  double p0 = 1.0, p1 = x;
  if (n == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  dP = n * (x * p1 - p0) / (x * x - 1.0);
}

static void gauss_rule(int nq, std::vector<double>& x, std::vector<double>& w) {
  // nq-point Gauss-Legendre on [0,1]
  x.resize(nq);
  w.resize(nq);
  for (int i = 0; i < nq; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (nq + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_pd(nq, t, P, dP);
      double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double P, dP;
    legendre_pd(nq, t, P, dP);
    x[i] = 0.5 * (1.0 - t);
    w[i] = 1.0 / ((1.0 - t * t) * dP * dP);  // (2 / ((1-t^2) P'^2)) / 2
  }
}

static std::vector<double> gll_nodes(int p) {
  std::vector<double> x(p + 1);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_pd(p, t, P, dP);
      double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      double dt = dP / d2P;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  std::sort(x.begin(), x.end());
  for (auto& v : x) v = 0.5 * (v + 1.0);
  return x;
}

static double lagrange_value(const std::vector<double>& nodes, int a, double x) {
  double v = 1.0;
  for (size_t b = 0; b < nodes.size(); ++b)
    if ((int)b != a) v *= (x - nodes[b]) / (nodes[a] - nodes[b]);
  return v;
}

Ref1D reference_1d(int p) {
  Ref1D r;
  r.p = p;
  r.nodes = gll_nodes(p);
  const int np = p + 1;
  // barycentric weights and the nodal differentiation matrix D[i][j] = l_j'(x_i)
  std::vector<double> lam(np, 1.0);
  for (int j = 0; j < np; ++j)
    for (int k = 0; k < np; ++k)
      if (k != j) lam[j] /= (r.nodes[j] - r.nodes[k]);
  std::vector<double> D(np * np, 0.0);
  for (int i = 0; i < np; ++i) {
    double s = 0.0;
    for (int j = 0; j < np; ++j)
      if (j != i) {
        D[i * np + j] = (lam[j] / lam[i]) / (r.nodes[i] - r.nodes[j]);
        s += D[i * np + j];
      }
    D[i * np + i] = -s;
  }
  std::vector<double> xq, wq;
  gauss_rule(p + 2, xq, wq);  // exact for degree 2p + 3
  const int nq = (int)xq.size();
  std::vector<double> V(nq * np), Vd(nq * np, 0.0);
  for (int q = 0; q < nq; ++q)
    for (int a = 0; a < np; ++a) V[q * np + a] = lagrange_value(r.nodes, a, xq[q]);
  // l_a'(x_q) = sum_i l_i(x_q) D[i][a]  (l_a' has degree p-1, interpolated exactly)
  for (int q = 0; q < nq; ++q)
    for (int a = 0; a < np; ++a) {
      double s = 0.0;
      for (int i = 0; i < np; ++i) s += V[q * np + i] * D[i * np + a];
      Vd[q * np + a] = s;
    }
  r.M.assign(np * np, 0.0);
  r.K.assign(np * np, 0.0);
  for (int a = 0; a < np; ++a)
    for (int b = 0; b < np; ++b) {
      double sm = 0.0, sk = 0.0;
      for (int q = 0; q < nq; ++q) {
        sm += wq[q] * V[q * np + a] * V[q * np + b];
        sk += wq[q] * Vd[q * np + a] * Vd[q * np + b];
      }
      r.M[a * np + b] = sm;
      r.K[a * np + b] = sk;
    }
  // degree-p/2 interpolation through p/2+1 equispaced points, evaluated at the GLL nodes
  const int q = p / 2;
  std::vector<double> eq(q + 1);
  for (int b = 0; b <= q; ++b) eq[b] = (double)b / q;
  r.Pw.assign(np * (q + 1), 0.0);
  for (int a = 0; a < np; ++a)
    for (int b = 0; b <= q; ++b) r.Pw[a * (q + 1) + b] = lagrange_value(eq, b, r.nodes[a]);
  // exact end-point values (Lagrange property at shared vertices)
  for (int b = 0; b <= q; ++b) {
    r.Pw[0 * (q + 1) + b] = (b == 0) ? 1.0 : 0.0;
    r.Pw[p * (q + 1) + b] = (b == q) ? 1.0 : 0.0;
  }
  return r;
}

// --------------------------------------------------------------- partition
Block1D partition_1d(int n, int l_dd) {
  Block1D b;
  int nb = (n + l_dd - 1) / l_dd;
  int base = n / nb, rem = n % nb;
  int s = 0;
  for (int i = 0; i < nb; ++i) {
    int z = base + (i < rem ? 1 : 0);
    b.start.push_back(s);
    b.size.push_back(z);
    s += z;
  }
  return b;
}

th_status make_geometry(const th_mesh& mesh, const th_params& prm, Geometry& g) {
  if (mesh.dim != 2 && mesh.dim != 3) return TH_ERR_UNSUPPORTED;
  if (mesh.n < 1 || mesh.n > (mesh.dim == 3 ? 256 : 4096)) return TH_ERR_ARG;
  if (mesh.p < 2 || mesh.p > kMaxP || (mesh.p % 2) != 0) return TH_ERR_ARG;
  if (mesh.dim == 3 && mesh.p != 2) return TH_ERR_UNSUPPORTED;  // the 3-D kernels are Q2
  const int nsides = 2 * mesh.dim;
  for (int s = 0; s < nsides; ++s) {
    if (mesh.bc[s] == TH_BC_DIRICHLET && mesh.dim == 3) return TH_ERR_UNSUPPORTED;  // 2-D only
    if (mesh.bc[s] != TH_BC_ROBIN && mesh.bc[s] != TH_BC_NEUMANN && mesh.bc[s] != TH_BC_DIRICHLET)
      return TH_ERR_ARG;
  }
  if (prm.l_dd < 1 || prm.n_dd < 1 || prm.n_s < 1) return TH_ERR_ARG;
  if (prm.restart < 1 || prm.maxit < 0 || prm.nrhs_max < 1 || prm.nrhs_max > 4096) return TH_ERR_ARG;
  if (prm.prec < TH_PREC_FP64 || prm.prec > TH_PREC_FP16) return TH_ERR_ARG;
  if (!(prm.tol >= 0.0) || !std::isfinite(prm.alpha_s) || !std::isfinite(prm.omega_c)) return TH_ERR_ARG;
  g.dim = mesh.dim;
  g.n = mesh.n;
  g.p = mesh.p;
  g.q = mesh.p / 2;
  g.m = g.n * g.p + 1;
  g.nc = g.n * g.q;
  g.mc = g.nc + 1;
  g.N = g.Nc = 1;
  for (int d = 0; d < g.dim; ++d) {
    g.N *= g.m;
    g.Nc *= g.mc;
  }
  g.h = 1.0 / g.n;
  g.hc = 1.0 / g.nc;
  for (int s = 0; s < 6; ++s) g.robin[s] = (s < nsides && mesh.bc[s] == TH_BC_ROBIN) ? 1 : 0;
  for (int s = 0; s < 6; ++s) g.dirichlet[s] = (s < nsides && mesh.bc[s] == TH_BC_DIRICHLET) ? 1 : 0;
  g.l_dd = std::min(prm.l_dd, g.n);
  g.blk = partition_1d(g.n, g.l_dd);
  g.nb = (int)g.blk.start.size();
  const int nbz = g.dim == 3 ? g.nb : 1;
  g.nsub = g.nb * g.nb * nbz;
  int lmax = *std::max_element(g.blk.size.begin(), g.blk.size.end());
  g.Lu = lmax * g.p + 1;
  g.Lw = std::min(lmax + 2, g.n) * g.p + 1;
  g.NR = g.Lu * g.Lu * (g.dim == 3 ? g.Lu : 1);
  g.NC = g.Lw * g.Lw * (g.dim == 3 ? g.Lw : 1);
  // boxes
  std::vector<int> o0(g.nb), o1(g.nb);
  for (int b = 0; b < g.nb; ++b) {
    o0[b] = std::max(g.blk.start[b] - 1, 0);
    o1[b] = std::min(g.blk.start[b] + g.blk.size[b] + 1, g.n);
  }
  g.box.resize((size_t)g.nsub * kBox);
  for (int bz = 0; bz < nbz; ++bz)
    for (int by = 0; by < g.nb; ++by)
      for (int bx = 0; bx < g.nb; ++bx) {
        int* bb = &g.box[(((size_t)bz * g.nb + by) * g.nb + bx) * kBox];
        bb[0] = o0[bx] * g.p;
        bb[1] = o0[by] * g.p;
        bb[2] = (o1[bx] - o0[bx]) * g.p + 1;
        bb[3] = (o1[by] - o0[by]) * g.p + 1;
        bb[4] = g.blk.start[bx] * g.p;
        bb[5] = g.blk.start[by] * g.p;
        bb[6] = g.blk.size[bx] * g.p + 1;
        bb[7] = g.blk.size[by] * g.p + 1;
        if (g.dim == 3) {
          bb[8] = o0[bz] * g.p;
          bb[9] = (o1[bz] - o0[bz]) * g.p + 1;
          bb[10] = g.blk.start[bz] * g.p;
          bb[11] = g.blk.size[bz] * g.p + 1;
        } else {
          bb[8] = 0;
          bb[9] = 1;
          bb[10] = 0;
          bb[11] = 1;
        }
      }
  // 1-D combine table and multiplicity
  g.ctab.assign((size_t)g.m * 4, -1);
  g.mult1d.assign(g.m, 0);
  for (int b = 0; b < g.nb; ++b) {
    int lo = g.blk.start[b] * g.p, hi = (g.blk.start[b] + g.blk.size[b]) * g.p;
    for (int i = lo; i <= hi; ++i) {
      int c = g.mult1d[i]++;
      g.ctab[(size_t)i * 4 + 2 * c] = b;
      g.ctab[(size_t)i * 4 + 2 * c + 1] = i - lo;
    }
  }
  return TH_OK;
}

// ------------------------------------------------------ subdomain matrices
// Banded LU with partial pivoting on dense row-major storage (LAPACK gbtrf
// semantics: the interchange of step k is applied to the right-hand side
// just before the elimination of step k).
static bool band_lu(cplx* A, int n, int kl, int ku, std::vector<int>& piv) {
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int rmax = std::min(n - 1, k + kl);
    int pr = k;
    double best = std::abs(A[(size_t)k * n + k]);
    for (int r = k + 1; r <= rmax; ++r) {
      double v = std::abs(A[(size_t)r * n + k]);
      if (v > best) { best = v; pr = r; }
    }
    if (best == 0.0) return false;
    piv[k] = pr;
    int cmax = std::min(n - 1, k + kl + ku);
    if (pr != k)
      for (int c = k; c <= cmax; ++c) std::swap(A[(size_t)k * n + c], A[(size_t)pr * n + c]);
    cplx inv = 1.0 / A[(size_t)k * n + k];
    const cplx* rowk = A + (size_t)k * n;
    for (int r = k + 1; r <= rmax; ++r) {
      cplx* rowr = A + (size_t)r * n;
      cplx l = rowr[k] * inv;
      rowr[k] = l;
      if (l == 0.0) continue;
      for (int c = k + 1; c <= cmax; ++c) rowr[c] -= l * rowk[c];
    }
  }
  return true;
}

static void band_solve(const cplx* A, int n, int kl, int ku, const std::vector<int>& piv, cplx* b) {
  for (int k = 0; k < n; ++k) {
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
    cplx bk = b[k];
    if (bk == 0.0) continue;
    int rmax = std::min(n - 1, k + kl);
    for (int r = k + 1; r <= rmax; ++r) b[r] -= A[(size_t)r * n + k] * bk;
  }
  for (int k = n - 1; k >= 0; --k) {
    int cmax = std::min(n - 1, k + kl + ku);
    cplx s = b[k];
    for (int c = k + 1; c <= cmax; ++c) s -= A[(size_t)k * n + c] * b[c];
    b[k] = s / A[(size_t)k * n + k];
  }
}

// 3-D: Omega^(i) box of wx x wy x wz dofs; element matrices
// h (K M M + M K M + M M K) - (k^2 (1 + i a) + i eps) h^3 M M M, and
// -i k h^2 M M on every absorbing face (internal faces of Omega^(i) and the
// domain's Robin faces), lexicographic local numbering, x fastest.
static th_status subdomain_inverse_rows3(const Geometry& g, const Ref1D& ref, const double* k,
                                         const double* eps, double alpha_s, int sub, cplx* out) {
  const int* bb = &g.box[(size_t)sub * kBox];
  const int ox = bb[0], oy = bb[1], wx = bb[2], wy = bb[3];
  const int ux = bb[4], uy = bb[5], vx = bb[6], vy = bb[7];
  const int oz = bb[8], wz = bb[9], uz = bb[10], vz = bb[11];
  const int p = g.p, np = p + 1;
  const int nx = (wx - 1) / p, ny = (wy - 1) / p, nz = (wz - 1) / p;
  const int c0x = ox / p, c0y = oy / p, c0z = oz / p;
  const int nd = wx * wy * wz;
  std::vector<cplx> A((size_t)nd * nd, 0.0);
  const double h = g.h;
  const double* M = ref.M.data();
  const double* K = ref.K.data();
  auto lid = [&](int lz, int ly, int lx) { return (lz * wy + ly) * wx + lx; };
  for (int cz = 0; cz < nz; ++cz)
    for (int cy = 0; cy < ny; ++cy)
      for (int cx = 0; cx < nx; ++cx) {
        const size_t cell = ((size_t)(c0z + cz) * g.n + (c0y + cy)) * g.n + (c0x + cx);
        const double kk = k[cell], ee = eps ? eps[cell] : 0.0;
        const cplx me = -cplx(kk * kk, alpha_s * kk * kk + ee) * (h * h * h);
        for (int az = 0; az < np; ++az)
          for (int ay = 0; ay < np; ++ay)
            for (int ax = 0; ax < np; ++ax) {
              const int row = lid(cz * p + az, cy * p + ay, cx * p + ax);
              for (int bz = 0; bz < np; ++bz)
                for (int by = 0; by < np; ++by)
                  for (int bx = 0; bx < np; ++bx) {
                    const int col = lid(cz * p + bz, cy * p + by, cx * p + bx);
                    const double Mz = M[az * np + bz], My = M[ay * np + by], Mx = M[ax * np + bx];
                    const double st = K[az * np + bz] * My * Mx + Mz * K[ay * np + by] * Mx + Mz * My * K[ax * np + bx];
                    A[(size_t)row * nd + col] += h * st + me * (Mz * My * Mx);
                  }
            }
      }
  // absorbing faces: side s = 2 axis + end, axis 0 = x, 1 = y, 2 = z
  const int ncl[3] = {nx, ny, nz}, c0[3] = {c0x, c0y, c0z}, wl[3] = {wx, wy, wz};
  for (int s = 0; s < 6; ++s) {
    const int ax = s / 2, end = s % 2;
    const bool at_domain = end == 0 ? (c0[ax] == 0) : (c0[ax] + ncl[ax] == g.n);
    if (at_domain && !g.robin[s]) continue;
    const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;  // the face's two axes
    const int layer = end == 0 ? 0 : wl[ax] - 1;
    for (int f2 = 0; f2 < ncl[a2]; ++f2)
      for (int f1 = 0; f1 < ncl[a1]; ++f1) {
        int cc[3];
        cc[ax] = end == 0 ? 0 : ncl[ax] - 1;
        cc[a1] = f1;
        cc[a2] = f2;
        const size_t cell = ((size_t)(c0z + cc[2]) * g.n + (c0y + cc[1])) * g.n + (c0x + cc[0]);
        const cplx rho(0.0, -k[cell] * h * h);  // -i k h^2
        for (int i2 = 0; i2 < np; ++i2)
          for (int i1 = 0; i1 < np; ++i1)
            for (int j2 = 0; j2 < np; ++j2)
              for (int j1 = 0; j1 < np; ++j1) {
                int ra[3], rb[3];
                ra[ax] = rb[ax] = layer;
                ra[a1] = f1 * p + i1;
                ra[a2] = f2 * p + i2;
                rb[a1] = f1 * p + j1;
                rb[a2] = f2 * p + j2;
                A[(size_t)lid(ra[2], ra[1], ra[0]) * nd + lid(rb[2], rb[1], rb[0])] +=
                    rho * (M[i1 * np + j1] * M[i2 * np + j2]);
              }
      }
  }
  const int bw = p * wx * wy + p * wx + p;
  std::vector<int> piv;
  if (!band_lu(A.data(), nd, bw, bw, piv)) return TH_ERR_SINGULAR;
  std::vector<cplx> x(nd);
  const int NC = g.NC, Lu = g.Lu, Lw = g.Lw;
  std::fill(out, out + (size_t)g.NR * NC, cplx(0.0));
  for (int rz = 0; rz < vz; ++rz)
    for (int ry = 0; ry < vy; ++ry)
      for (int rx = 0; rx < vx; ++rx) {
        const int gx = ux + rx, gy = uy + ry, gz = uz + rz;
        std::fill(x.begin(), x.end(), cplx(0.0));
        x[lid(gz - oz, gy - oy, gx - ox)] = 1.0;
        band_solve(A.data(), nd, bw, bw, piv, x.data());
        const double Lj = (double)g.mult1d[gx] * g.mult1d[gy] * g.mult1d[gz];
        cplx* orow = out + (size_t)((rz * Lu + ry) * Lu + rx) * NC;
        for (int cz = 0; cz < wz; ++cz)
          for (int cy = 0; cy < wy; ++cy)
            for (int cx = 0; cx < wx; ++cx) orow[(cz * Lw + cy) * Lw + cx] = x[lid(cz, cy, cx)] / Lj;
      }
  return TH_OK;
}

th_status subdomain_inverse_rows(const Geometry& g, const Ref1D& ref, const double* k,
                                 const double* eps, double alpha_s, int sub, cplx* out) {
  if (g.dim == 3) return subdomain_inverse_rows3(g, ref, k, eps, alpha_s, sub, out);
  const int* bb = &g.box[(size_t)sub * kBox];
  const int ox = bb[0], oy = bb[1], wx = bb[2], wy = bb[3];
  const int ux = bb[4], uy = bb[5], vx = bb[6], vy = bb[7];
  const int p = g.p, np = p + 1;
  const int ncx = (wx - 1) / p, ncy = (wy - 1) / p;
  const int c0x = ox / p, c0y = oy / p;
  const int nd = wx * wy;
  std::vector<cplx> A((size_t)nd * nd, 0.0);
  const double h = g.h;
  // volume terms: stiffness K(x)M(y) + M(x)K(y), shifted mass -(k^2 (1 + i a) + i eps) h^2 M M
  for (int cy = 0; cy < ncy; ++cy)
    for (int cx = 0; cx < ncx; ++cx) {
      const size_t cell = (size_t)(c0y + cy) * g.n + (c0x + cx);
      const double kk = k[cell], ee = eps ? eps[cell] : 0.0;
      const cplx me = -cplx(kk * kk, alpha_s * kk * kk + ee) * (h * h);
      for (int ay = 0; ay < np; ++ay)
        for (int ax = 0; ax < np; ++ax) {
          const int row = (cy * p + ay) * wx + cx * p + ax;
          for (int by = 0; by < np; ++by)
            for (int bx = 0; bx < np; ++bx) {
              const int col = (cy * p + by) * wx + cx * p + bx;
              const double mm = ref.M[ay * np + by] * ref.M[ax * np + bx];
              const double st = ref.M[ay * np + by] * ref.K[ax * np + bx] + ref.K[ay * np + by] * ref.M[ax * np + bx];
              A[(size_t)row * nd + col] += st + me * mm;
            }
        }
    }
  // absorbing sides: internal sides of Omega^(i), and Robin sides of the domain
  const bool at_lo_x = (c0x == 0), at_hi_x = (c0x + ncx == g.n);
  const bool at_lo_y = (c0y == 0), at_hi_y = (c0y + ncy == g.n);
  const bool side_abs[4] = {at_lo_x ? (bool)g.robin[0] : true, at_hi_x ? (bool)g.robin[1] : true,
                            at_lo_y ? (bool)g.robin[2] : true, at_hi_y ? (bool)g.robin[3] : true};
  for (int s = 0; s < 4; ++s) {
    if (!side_abs[s]) continue;
    const bool xside = (s < 2);
    const int ncell = xside ? ncy : ncx;
    for (int c = 0; c < ncell; ++c) {
      int cx, cy;
      if (xside) { cy = c; cx = (s == 0) ? 0 : ncx - 1; }
      else { cx = c; cy = (s == 2) ? 0 : ncy - 1; }
      const size_t cell = (size_t)(c0y + cy) * g.n + (c0x + cx);
      const cplx rho(0.0, -k[cell] * h);  // -i k h
      for (int a = 0; a < np; ++a)
        for (int b = 0; b < np; ++b) {
          int ra, rb;
          if (xside) {
            const int lx = (s == 0) ? 0 : wx - 1;
            ra = (cy * p + a) * wx + lx;
            rb = (cy * p + b) * wx + lx;
          } else {
            const int ly = (s == 2) ? 0 : wy - 1;
            ra = ly * wx + cx * p + a;
            rb = ly * wx + cx * p + b;
          }
          A[(size_t)ra * nd + rb] += rho * ref.M[a * np + b];
        }
    }
  }
  // Dirichlet sides of the domain in this subdomain's boundary (Gamma_0, inherited):
  // the unknowns there are decoupled, identity rows and columns
  {
    const bool dside[4] = {at_lo_x && g.dirichlet[0], at_hi_x && g.dirichlet[1], at_lo_y && g.dirichlet[2],
                           at_hi_y && g.dirichlet[3]};
    if (dside[0] || dside[1] || dside[2] || dside[3]) {
      std::vector<char> dn(nd, 0);
      for (int ly = 0; ly < wy; ++ly)
        for (int lx = 0; lx < wx; ++lx)
          if ((dside[0] && lx == 0) || (dside[1] && lx == wx - 1) || (dside[2] && ly == 0) ||
              (dside[3] && ly == wy - 1))
            dn[(size_t)ly * wx + lx] = 1;
      for (int i = 0; i < nd; ++i) {
        if (!dn[i]) continue;
        for (int j = 0; j < nd; ++j) {
          A[(size_t)i * nd + j] = 0.0;
          A[(size_t)j * nd + i] = 0.0;
        }
        A[(size_t)i * nd + i] = 1.0;
      }
    }
  }
  // banded LU: coupling within a cell reaches p rows and p columns
  const int bw = p * wx + p;
  std::vector<int> piv;
  if (!band_lu(A.data(), nd, bw, bw, piv)) return TH_ERR_SINGULAR;
  // A_s^(i) is complex symmetric, so row j of its inverse solves A x = e_j.
  std::vector<cplx> x(nd);
  const int NR = g.NR, NC = g.NC, Lu = g.Lu, Lw = g.Lw;
  std::fill(out, out + (size_t)NR * NC, cplx(0.0));
  for (int ry = 0; ry < vy; ++ry)
    for (int rx = 0; rx < vx; ++rx) {
      const int gx = ux + rx, gy = uy + ry;
      const int lj = (gy - oy) * wx + (gx - ox);
      std::fill(x.begin(), x.end(), cplx(0.0));
      x[lj] = 1.0;
      band_solve(A.data(), nd, bw, bw, piv, x.data());
      const double Lj = (double)g.mult1d[gx] * g.mult1d[gy];
      cplx* orow = out + (size_t)(ry * Lu + rx) * NC;
      for (int cy = 0; cy < wy; ++cy)
        for (int cx = 0; cx < wx; ++cx) orow[cy * Lw + cx] = x[cy * wx + cx] / Lj;
    }
  return TH_OK;
}

th_status all_inverse_rows(const Geometry& g, const Ref1D& ref, const double* k, const double* eps,
                           double alpha_s, std::vector<cplx>& out) {
  const size_t blk = (size_t)g.NR * g.NC;
  out.assign(blk * g.nsub, cplx(0.0));
  // identical subdomains (same boxes relative to the boundary, same coefficients,
  // same multiplicities) give identical rows: compute each distinct one once
  std::vector<int> rep(g.nsub);
  std::map<std::string, int> seen;
  for (int s = 0; s < g.nsub; ++s) {
    const int* bb = &g.box[(size_t)s * kBox];
    std::string key;
    auto put = [&](const void* d, size_t nbytes) { key.append((const char*)d, nbytes); };
    const int ox = bb[0], oy = bb[1], wx = bb[2], wy = bb[3], oz = bb[8], wz = bb[9];
    int rel[12] = {bb[2], bb[3], bb[4] - ox, bb[5] - oy, bb[6], bb[7],
                   (ox == 0) ? 1 : 0, (oy == 0) ? 1 : 0, bb[9], bb[10] - oz, bb[11], (oz == 0) ? 1 : 0};
    put(rel, sizeof(rel));
    int hi[3] = {(ox + wx - 1 == g.m - 1) ? 1 : 0, (oy + wy - 1 == g.m - 1) ? 1 : 0,
                 (g.dim == 3 && oz + wz - 1 == g.m - 1) ? 1 : 0};
    put(hi, sizeof(hi));
    const int czb = g.dim == 3 ? oz / g.p : 0, cze = g.dim == 3 ? (oz + wz - 1) / g.p : 1;
    for (int cz = czb; cz < cze; ++cz)
      for (int cy = oy / g.p; cy < (oy + wy - 1) / g.p; ++cy)
        for (int cx = ox / g.p; cx < (ox + wx - 1) / g.p; ++cx) {
          const size_t c = ((size_t)cz * g.n + cy) * g.n + cx;
          put(&k[c], sizeof(double));
          double e = eps ? eps[c] : 0.0;
          put(&e, sizeof(double));
        }
    for (int i = bb[4]; i < bb[4] + bb[6]; ++i) put(&g.mult1d[i], sizeof(int));
    for (int i = bb[5]; i < bb[5] + bb[7]; ++i) put(&g.mult1d[i], sizeof(int));
    if (g.dim == 3)
      for (int i = bb[10]; i < bb[10] + bb[11]; ++i) put(&g.mult1d[i], sizeof(int));
    auto it = seen.find(key);
    if (it == seen.end()) {
      seen.emplace(key, s);
      rep[s] = s;
    } else {
      rep[s] = it->second;
    }
  }
  std::vector<int> todo;
  for (int s = 0; s < g.nsub; ++s)
    if (rep[s] == s) todo.push_back(s);
  std::atomic<int> err(0);
  parallel_for((int)todo.size(), [&](int i) {
    int s = todo[i];
    th_status st = subdomain_inverse_rows(g, ref, k, eps, alpha_s, s, out.data() + blk * s);
    if (st != TH_OK) err.store((int)st);
  });
  if (err.load() != 0) return (th_status)err.load();
  for (int s = 0; s < g.nsub; ++s)
    if (rep[s] != s) std::copy(out.begin() + blk * rep[s], out.begin() + blk * (rep[s] + 1), out.begin() + blk * s);
  return TH_OK;
}

// -------------------------------------------------------------------- QSFEM
// The printed formulas for P1, P2 and N are ratios of quantities that all
// vanish as eta -> 0 (numerators and denominator like eta^4, sigma_P(0) den
// like eta^6), so evaluating them as written loses about eta^-6 ulps.  Each
// quantity is a signed sum of cosines sum_j w_j cos(eta t_j) (products of
// cosines turned into sums), and its low Taylor moments sum_j w_j t_j^(2k)
// vanish exactly (k = 0, 1 for the numerators and the denominator, k = 0, 1, 2
// for E = 4 den + 8 num1 + 4 num2 = den sigma_P(0)).  The sums are therefore
// evaluated with the remainders cos x - 1 + x^2/2 (resp. - x^4/24 too), which
// carry no cancellation.  Then
//   q00 = N P0/4 = -eta^2 den / E,  q_edge = N P1/2 = -eta^2 num1 / E,
//   q_diag = N P2 = -eta^2 num2 / E.
static double cos_rem(double x, int order) {
  // order 4: cos x - 1 + x^2/2;  order 6: cos x - 1 + x^2/2 - x^4/24
  const double ax = std::fabs(x);
  if (ax > 1.5) {
    double v = std::cos(x) - 1.0 + 0.5 * x * x;
    if (order == 6) v -= x * x * x * x / 24.0;
    return v;
  }
  const double x2 = x * x;
  double term = (order == 4) ? x2 * x2 / 24.0 : -x2 * x2 * x2 / 720.0;  // first term
  int k = (order == 4) ? 2 : 3;
  double sum = 0.0;
  for (int it = 0; it < 20; ++it) {
    sum += term;
    term *= -x2 / ((2.0 * k + 1.0) * (2.0 * k + 2.0));
    ++k;
  }
  return sum;
}

void qsfem_cell(double k, double eps, double hc, cplx d[3]) {
  const double eta = k * hc;
  const double a = std::cos(M_PI / 16), b = std::sin(M_PI / 16);
  const double c = std::cos(3 * M_PI / 16), e = std::sin(3 * M_PI / 16);
  struct Term { double w, t; };
  // num1 = c1 s1 - c2 s2, num2 = c2 + s2 - c1 - s1, den = c2 s2 (c1 + s1) - c1 s1 (c2 + s2)
  const Term n1[4] = {{0.5, a + b}, {0.5, a - b}, {-0.5, c + e}, {-0.5, c - e}};
  const Term n2[4] = {{1, c}, {1, e}, {-1, a}, {-1, b}};
  Term dn[16];
  const double trip[4][4] = {{c, e, a, 1}, {c, e, b, 1}, {a, b, c, -1}, {a, b, e, -1}};
  for (int i = 0; i < 4; ++i) {
    const double x = trip[i][0], y = trip[i][1], z = trip[i][2], w = 0.25 * trip[i][3];
    dn[4 * i + 0] = {w, x + y + z};
    dn[4 * i + 1] = {w, x + y - z};
    dn[4 * i + 2] = {w, x - y + z};
    dn[4 * i + 3] = {w, x - y - z};
  }
  double num1 = 0, num2 = 0, den = 0, E = 0;
  for (const Term& t : n1) { num1 += t.w * cos_rem(eta * t.t, 4); E += 8 * t.w * cos_rem(eta * t.t, 6); }
  for (const Term& t : n2) { num2 += t.w * cos_rem(eta * t.t, 4); E += 4 * t.w * cos_rem(eta * t.t, 6); }
  for (const Term& t : dn) { den += t.w * cos_rem(eta * t.t, 4); E += 4 * t.w * cos_rem(eta * t.t, 6); }
  const double s = -eta * eta / E;
  const double h2 = hc * hc;
  d[0] = cplx(s * den, -eps * h2 / 9.0);
  d[1] = cplx(s * num1, -eps * h2 / 18.0);
  d[2] = cplx(s * num2, -eps * h2 / 36.0);
}

static bool dense_inverse_par(std::vector<cplx>& S, int n, cplx* out);

// Inverse of a dense complex matrix (LU with partial pivoting, then one
// triangular solve per unit column, columns in parallel); for n >= 1024 the
// LU's trailing update is split over a thread team (dense_inverse_par: the same
// operations in the same order, so the same result; for the 2-D coarse blocks,
// n <= 1024, its two team barriers per pivot cost more than they save: 40 s
// against 18 s for the 401 blocks of 401 rows).  Callers outside a parallel region.
static bool dense_inverse(std::vector<cplx>& S, int n, cplx* out) {
  if (n >= 1024) return dense_inverse_par(S, n, out);
  std::vector<int> piv;
  if (!band_lu(S.data(), n, n - 1, n - 1, piv)) return false;
  // column c of the inverse solves S x = e_c; write it as column c of out
  parallel_for(n, [&](int c) {
    std::vector<cplx> x(n, cplx(0.0));
    x[c] = 1.0;
    band_solve(S.data(), n, n - 1, n - 1, piv, x.data());
    for (int r = 0; r < n; ++r) out[(size_t)r * n + c] = x[r];
  });
  return true;
}

th_status coarse_setup(const Geometry& g, const double* k, const double* eps, CoarseBlocks& cb,
                       bool block_inverses) {
  const int nc = g.nc, mc = g.mc, q = g.q;
  cb.mc = mc;
  cb.cell.assign((size_t)nc * nc * 3, cplx(0.0));
  for (int cy = 0; cy < nc; ++cy)
    for (int cx = 0; cx < nc; ++cx) {
      const size_t f = (size_t)(cy / q) * g.n + (cx / q);
      qsfem_cell(k[f], eps ? eps[f] : 0.0, g.hc, &cb.cell[((size_t)cy * nc + cx) * 3]);
    }
  for (int s = 0; s < 4; ++s) {
    cb.rho[s].assign(nc, cplx(0.0));
    if (!g.robin[s]) continue;
    for (int t = 0; t < nc; ++t) {
      int cx, cy;
      if (s < 2) { cy = t; cx = (s == 0) ? 0 : nc - 1; }
      else { cx = t; cy = (s == 2) ? 0 : nc - 1; }
      const size_t f = (size_t)(cy / q) * g.n + (cx / q);
      cb.rho[s][t] = cplx(0.0, -k[f] * g.hc);
    }
  }
  const size_t mm = (size_t)mc * mc;
  cb.dl.assign(mm, 0.0); cb.dd.assign(mm, 0.0); cb.du.assign(mm, 0.0);
  cb.cl.assign(mm, 0.0); cb.cd.assign(mm, 0.0); cb.cu.assign(mm, 0.0);
  auto add = [&](int ax, int ay, int bx, int by, cplx v) {
    // entry A[(ax,ay),(bx,by)] into the block structure (rows ay, lower blocks implied)
    const size_t r = (size_t)ay * mc + ax;
    const int dx = bx - ax;
    if (by == ay) {
      (dx == -1 ? cb.dl : dx == 0 ? cb.dd : cb.du)[r] += v;
    } else if (by == ay + 1) {
      (dx == -1 ? cb.cl : dx == 0 ? cb.cd : cb.cu)[r] += v;
    }
  };
  for (int cy = 0; cy < nc; ++cy)
    for (int cx = 0; cx < nc; ++cx) {
      const cplx* d = &cb.cell[((size_t)cy * nc + cx) * 3];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          const int ax = cx + (a & 1), ay = cy + (a >> 1);
          const int bx = cx + (b & 1), by = cy + (b >> 1);
          const int nd = std::abs(ax - bx) + std::abs(ay - by);
          add(ax, ay, bx, by, d[nd]);
        }
    }
  for (int s = 0; s < 4; ++s) {
    if (!g.robin[s]) continue;
    for (int t = 0; t < nc; ++t) {
      int x0, y0, x1, y1;
      if (s < 2) { x0 = x1 = (s == 0) ? 0 : nc; y0 = t; y1 = t + 1; }
      else { y0 = y1 = (s == 2) ? 0 : nc; x0 = t; x1 = t + 1; }
      const cplx r = cb.rho[s][t];
      add(x0, y0, x0, y0, r / 3.0);
      add(x1, y1, x1, y1, r / 3.0);
      add(x0, y0, x1, y1, r / 6.0);
      add(x1, y1, x0, y0, r / 6.0);
    }
  }
  // Dirichlet sides (Gamma_0): the coarse space vanishes there as well; the
  // coarse nodes on them are decoupled (identity rows, zero columns)
  for (int ay = 0; ay < mc; ++ay)
    for (int ax = 0; ax < mc; ++ax) {
      const bool dn = (g.dirichlet[0] && ax == 0) || (g.dirichlet[1] && ax == mc - 1) ||
                      (g.dirichlet[2] && ay == 0) || (g.dirichlet[3] && ay == mc - 1);
      if (!dn) continue;
      const size_t r = (size_t)ay * mc + ax;
      cb.dl[r] = cb.du[r] = 0.0;
      cb.dd[r] = 1.0;
      cb.cl[r] = cb.cd[r] = cb.cu[r] = 0.0;          // row r's couplings to block row ay + 1
      if (ax > 0) cb.du[r - 1] = 0.0;                  // column r in block row ay
      if (ax + 1 < mc) cb.dl[r + 1] = 0.0;
      if (ay > 0) {                                    // column r in C_{ay-1} (and so in B_ay)
        const size_t o = (size_t)(ay - 1) * mc;
        cb.cd[o + ax] = 0.0;
        if (ax > 0) cb.cu[o + ax - 1] = 0.0;
        if (ax + 1 < mc) cb.cl[o + ax + 1] = 0.0;
      }
    }
  // block elimination: S_0 = D_0, S_j = D_j - B_j S_{j-1}^{-1} C_{j-1}, B_j = C_{j-1}^T
  if (!block_inverses) return TH_OK;
  cb.G.assign((size_t)mc * mm, cplx(0.0));
  std::vector<cplx> S(mm), T(mm);
  for (int j = 0; j < mc; ++j) {
    std::fill(S.begin(), S.end(), cplx(0.0));
    const size_t o = (size_t)j * mc;
    for (int a = 0; a < mc; ++a) {
      if (a > 0) S[(size_t)a * mc + a - 1] = cb.dl[o + a];
      S[(size_t)a * mc + a] = cb.dd[o + a];
      if (a + 1 < mc) S[(size_t)a * mc + a + 1] = cb.du[o + a];
    }
    if (j > 0) {
      const cplx* Gp = &cb.G[(size_t)(j - 1) * mm];
      const size_t op = (size_t)(j - 1) * mc;
      // T = G_{j-1} C_{j-1}:  T[a][b] = G[a][b-1] cu[b-1] + G[a][b] cd[b] + G[a][b+1] cl[b+1]
      parallel_for(mc, [&](int a) {
        for (int b = 0; b < mc; ++b) {
          cplx s = Gp[(size_t)a * mc + b] * cb.cd[op + b];
          if (b > 0) s += Gp[(size_t)a * mc + b - 1] * cb.cu[op + b - 1];
          if (b + 1 < mc) s += Gp[(size_t)a * mc + b + 1] * cb.cl[op + b + 1];
          T[(size_t)a * mc + b] = s;
        }
      });
      // S -= B_j T with B_j[a][a-1] = cu[a-1], B_j[a][a] = cd[a], B_j[a][a+1] = cl[a+1]
      parallel_for(mc, [&](int a) {
        for (int b = 0; b < mc; ++b) {
          cplx s = cb.cd[op + a] * T[(size_t)a * mc + b];
          if (a > 0) s += cb.cu[op + a - 1] * T[(size_t)(a - 1) * mc + b];
          if (a + 1 < mc) s += cb.cl[op + a + 1] * T[(size_t)(a + 1) * mc + b];
          S[(size_t)a * mc + b] -= s;
        }
      });
    }
    if (!dense_inverse(S, mc, &cb.G[(size_t)j * mm])) return TH_ERR_SINGULAR;
  }
  return TH_OK;
}

// ---------------------------------------------------------------- transfers
void transfer_tables(const Geometry& g, const Ref1D& ref, TransferTables& t) {
  const int p = g.p, q = g.q, m = g.m, mc = g.mc;
  t.q = q;
  t.pj0.assign(m, 0);
  t.pw.assign((size_t)m * (q + 1), 0.0);
  for (int i = 0; i < m; ++i) {
    int e = std::min(i / p, g.n - 1);
    int a = i - e * p;
    t.pj0[i] = e * q;
    for (int b = 0; b <= q; ++b) t.pw[(size_t)i * (q + 1) + b] = ref.Pw[a * (q + 1) + b];
  }
  // transpose: coarse node J collects every fine node with a nonzero weight on J
  std::vector<std::vector<std::pair<int, double>>> lists(mc);
  for (int i = 0; i < m; ++i)
    for (int b = 0; b <= q; ++b) {
      double w = t.pw[(size_t)i * (q + 1) + b];
      if (w != 0.0) lists[t.pj0[i] + b].push_back({i, w});
    }
  t.rmax = 0;
  for (auto& l : lists) t.rmax = std::max(t.rmax, (int)l.size());
  t.rcnt.assign(mc, 0);
  t.ridx.assign((size_t)mc * t.rmax, 0);
  t.rw.assign((size_t)mc * t.rmax, 0.0);
  for (int J = 0; J < mc; ++J) {
    t.rcnt[J] = (int)lists[J].size();
    for (size_t r = 0; r < lists[J].size(); ++r) {
      t.ridx[(size_t)J * t.rmax + r] = lists[J][r].first;
      t.rw[(size_t)J * t.rmax + r] = lists[J][r].second;
    }
    for (int r = (int)lists[J].size(); r < t.rmax; ++r) t.ridx[(size_t)J * t.rmax + r] = lists[J].empty() ? 0 : lists[J][0].first;
  }
}

// ------------------------------------------------ partitioned coarse solve
// The coarse rows are split into P chunks [a_c, b_c] separated by P - 1
// separator rows s_c = b_c + 1.  With y = A_cc^{-1} b_c (chunk c alone), the
// chunk rows of the solution are
//     x_j = y_j - L_j x_{s_{c-1}} - R_j x_{s_c},
//     L = A_cc^{-1} E_a B_a (left spike),  R = A_cc^{-1} E_b C_b (right spike),
// and the separators satisfy a block-tridiagonal system with P - 1 rows:
//     Shat_k x_k + What_k x_{k-1} + Ehat_k x_{k+1} = b_s - B_s y_{s-1} - C_s y_{s+1},
//     Shat_k = D_s - B_s R_{s-1} - C_s L_{s+1},  What_k = -B_s L_{s-1},  Ehat_k = -C_s R_{s+1},
// factorised as Ghat_k = (Shat_k - What_k Ghat_{k-1} Ehat_{k-1})^{-1}, F_k = Ghat_k What_k,
// H_k = Ghat_k Ehat_k.  Everything in FP64; dense blocks are stored with row stride mcp.
namespace {

using Mat = std::vector<cplx>;

// row i of C = alpha A B (+ C when acc), n x n dense row-major (k-j order)
inline void zgemm_row(int n, int i, const cplx* A, const cplx* B, cplx* C, cplx alpha, bool acc) {
  double* ci = reinterpret_cast<double*>(C + (size_t)i * n);
  if (!acc) std::fill(C + (size_t)i * n, C + (size_t)(i + 1) * n, cplx(0.0));
  for (int k = 0; k < n; ++k) {
    const cplx a = alpha * A[(size_t)i * n + k];
    const double ar = a.real(), ai = a.imag();
    if (ar == 0.0 && ai == 0.0) continue;
    const double* bk = reinterpret_cast<const double*>(B + (size_t)k * n);
    for (int j = 0; j < n; ++j) {
      const double br = bk[2 * j], bi = bk[2 * j + 1];
      ci[2 * j] += ar * br - ai * bi;
      ci[2 * j + 1] += ar * bi + ai * br;
    }
  }
}
// C = alpha A B (+ C when acc), serial
void zgemm(int n, const cplx* A, const cplx* B, cplx* C, cplx alpha, bool acc) {
  for (int i = 0; i < n; ++i) zgemm_row(n, i, A, B, C, alpha, acc);
}
// the same with the rows over threads (callers outside a parallel region)
void zgemm_par(int n, const cplx* A, const cplx* B, cplx* C, cplx alpha, bool acc) {
  parallel_for(n, [&](int i) { zgemm_row(n, i, A, B, C, alpha, acc); });
}

// Tridiagonal block helpers over the C_j diagonals (cl, cd, cu at row offset o = j mc):
// (C_j X)[a][:] = cl[a] X[a-1] + cd[a] X[a] + cu[a] X[a+1]
void tri_C_left(int n, const cplx* cl, const cplx* cd, const cplx* cu, const cplx* X, cplx* Y) {
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      cplx s = cd[a] * X[(size_t)a * n + b];
      if (a > 0) s += cl[a] * X[(size_t)(a - 1) * n + b];
      if (a + 1 < n) s += cu[a] * X[(size_t)(a + 1) * n + b];
      Y[(size_t)a * n + b] = s;
    }
}
// (B_{j+1} X) with B_{j+1} = C_j^T: row a = cu[a-1] X[a-1] + cd[a] X[a] + cl[a+1] X[a+1]
void tri_CT_left(int n, const cplx* cl, const cplx* cd, const cplx* cu, const cplx* X, cplx* Y) {
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      cplx s = cd[a] * X[(size_t)a * n + b];
      if (a > 0) s += cu[a - 1] * X[(size_t)(a - 1) * n + b];
      if (a + 1 < n) s += cl[a + 1] * X[(size_t)(a + 1) * n + b];
      Y[(size_t)a * n + b] = s;
    }
}
// Y = X C_j: Y[a][b] = X[a][b-1] cu[b-1] + X[a][b] cd[b] + X[a][b+1] cl[b+1]
void tri_C_right(int n, const cplx* cl, const cplx* cd, const cplx* cu, const cplx* X, cplx* Y) {
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      cplx s = X[(size_t)a * n + b] * cd[b];
      if (b > 0) s += X[(size_t)a * n + b - 1] * cu[b - 1];
      if (b + 1 < n) s += X[(size_t)a * n + b + 1] * cl[b + 1];
      Y[(size_t)a * n + b] = s;
    }
}
// Y = X C_j^T: Y[a][b] = X[a][b-1] cl[b] + X[a][b] cd[b] + X[a][b+1] cu[b]
void tri_CT_right(int n, const cplx* cl, const cplx* cd, const cplx* cu, const cplx* X, cplx* Y) {
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      cplx s = X[(size_t)a * n + b] * cd[b];
      if (b > 0) s += X[(size_t)a * n + b - 1] * cl[b];
      if (b + 1 < n) s += X[(size_t)a * n + b + 1] * cu[b];
      Y[(size_t)a * n + b] = s;
    }
}
bool zinverse_serial(int n, Mat& S, cplx* out) {
  std::vector<int> piv;
  if (!band_lu(S.data(), n, n - 1, n - 1, piv)) return false;
  std::vector<cplx> x(n);
  for (int c = 0; c < n; ++c) {
    std::fill(x.begin(), x.end(), cplx(0.0));
    x[c] = 1.0;
    band_solve(S.data(), n, n - 1, n - 1, piv, x.data());
    for (int r = 0; r < n; ++r) out[(size_t)r * n + c] = x[r];
  }
  return true;
}

void store_padded(int n, int ld, const cplx* M, cplx* dst) {
  for (int r = 0; r < n; ++r) std::copy(M + (size_t)r * n, M + (size_t)(r + 1) * n, dst + (size_t)r * ld);
}

}  // namespace


// -------------------------------------------------------------- 3-D coarse
// Fitted 27-point scheme (the paper only cites a 3-D dispersion-minimising
// stencil; this is the construction of the 9-point one carried to 3-D):
// sigma_P(xi) = P0 + 2 P1 sum cos xi_a + 4 P2 sum_{a<b} cos xi_a cos xi_b
// + 8 P3 prod cos xi_a vanishes at |xi| = eta along three directions d^(i)
// (images of the interior 3-point rule (2/3, 1/6, 1/6) of the symmetry-reduced
// spherical triangle with corners (0,0,1), (0,1,1)/sqrt2, (1,1,1)/sqrt3), and
// N = -eta^2 / sigma_P(0).  With s_a = 2 sin^2(eta d_a / 2) = 1 - cos(eta d_a)
// and S1 = sum s_a, S2 = sum_{a<b} s_a s_b, S3 = prod s_a, the zero conditions
// of the scaled weights read Q1 S1 - Q2 S2 + Q3 S3 = -eta^2, where
// Q1 = N (2 P1 + 8 P2 + 8 P3), Q2 = N (4 P2 + 8 P3), Q3 = 8 N P3.  Since
// S1 ~ eta^2, S2 ~ eta^4, S3 ~ eta^6, the system is solved for (Q1, eta^2 Q2,
// eta^4 Q3) with the columns divided by eta^2, eta^4, eta^6; Q2 and Q3 are then
// determined by the O(eta^4), O(eta^6) differences between the directions, so
// they lose about eta^-2 and eta^-4 units of the working precision, and the
// 3 x 3 solve runs in long double (the s_a are computed without cancellation).
// Then N P3 = Q3/8, N P2 = (Q2 - Q3)/4, N P1 = (Q1 - 2 Q2 + Q3)/2,
// N P0 = -eta^2 - 3 Q1 + 3 Q2 - Q3, and the cell's pair weights are
// h_c (N P0/8, N P1/4, N P2/2, N P3) minus i eps h_c^3 times the Q1 mass of
// the pair ((1/3)^(3 - nd) (1/6)^nd for nd differing coordinates).
void qsfem27_cell(double k, double eps, double hc, cplx d[4]) {
  static double dirs[3][3];
  static std::once_flag once;
  std::call_once(once, [] {
    const double r2 = 1.0 / std::sqrt(2.0), r3 = 1.0 / std::sqrt(3.0);
    const double V[3][3] = {{0, 0, 1}, {0, r2, r2}, {r3, r3, r3}};
    const double W[3][3] = {{2.0 / 3, 1.0 / 6, 1.0 / 6}, {1.0 / 6, 2.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 6, 2.0 / 3}};
    for (int i = 0; i < 3; ++i) {
      double v[3] = {0, 0, 0};
      for (int j = 0; j < 3; ++j)
        for (int a = 0; a < 3; ++a) v[a] += W[i][j] * V[j][a];
      const double nrm = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      for (int a = 0; a < 3; ++a) dirs[i][a] = v[a] / nrm;
    }
  });
  using L = long double;
  const L eta = (L)k * (L)hc, e2 = eta * eta;
  L Mx[3][4];
  for (int i = 0; i < 3; ++i) {
    L s[3];
    for (int a = 0; a < 3; ++a) {
      const L t = std::sin((L)0.5 * eta * (L)dirs[i][a]);
      s[a] = 2 * t * t;
    }
    const L S1 = s[0] + s[1] + s[2], S2 = s[0] * s[1] + s[0] * s[2] + s[1] * s[2], S3 = s[0] * s[1] * s[2];
    Mx[i][0] = S1 / e2;
    Mx[i][1] = -S2 / (e2 * e2);
    Mx[i][2] = S3 / (e2 * e2 * e2);
    Mx[i][3] = -1;  // right-hand side -eta^2 / eta^2
  }
  // Gaussian elimination with partial pivoting on the scaled 3 x 3 system
  for (int c = 0; c < 3; ++c) {
    int pr = c;
    for (int r = c + 1; r < 3; ++r)
      if (std::fabs(Mx[r][c]) > std::fabs(Mx[pr][c])) pr = r;
    for (int j = 0; j < 4; ++j) std::swap(Mx[c][j], Mx[pr][j]);
    for (int r = c + 1; r < 3; ++r) {
      const L l = Mx[r][c] / Mx[c][c];
      for (int j = c; j < 4; ++j) Mx[r][j] -= l * Mx[c][j];
    }
  }
  L y[3];
  for (int r = 2; r >= 0; --r) {
    L acc = Mx[r][3];
    for (int j = r + 1; j < 3; ++j) acc -= Mx[r][j] * y[j];
    y[r] = acc / Mx[r][r];
  }
  // unknowns were (Q1, eta^2 Q2, eta^4 Q3)
  const L Q1 = y[0], Q2 = y[1] / e2, Q3 = y[2] / (e2 * e2);
  const L NP3 = Q3 / 8, NP2 = (Q2 - Q3) / 4, NP1 = (Q1 - 2 * Q2 + Q3) / 2;
  const L NP0 = -e2 - 3 * Q1 + 3 * Q2 - Q3;
  const double q[4] = {(double)(NP0 / 8), (double)(NP1 / 4), (double)(NP2 / 2), (double)NP3};
  const double mass[4] = {1.0 / 27.0, 1.0 / 54.0, 1.0 / 108.0, 1.0 / 216.0};
  const double h3 = hc * hc * hc;
  for (int i = 0; i < 4; ++i) d[i] = cplx(hc * q[i], -eps * h3 * mass[i]);
}

namespace {
// Fixed-size thread team with a reusable barrier (host set-up only).
struct Team {
  int nt;
  std::mutex mu;
  std::condition_variable cv;
  int waiting = 0;
  long long gen = 0;
  explicit Team(int n) : nt(n) {}
  void barrier() {
    std::unique_lock<std::mutex> lk(mu);
    const long long g0 = gen;
    if (++waiting == nt) {
      waiting = 0;
      ++gen;
      cv.notify_all();
    } else {
      cv.wait(lk, [&] { return gen != g0; });
    }
  }
};
}  // namespace

// Inverse of a dense n x n matrix: right-looking LU with partial pivoting whose
// trailing update is split row-wise over a thread team, then the columns of
// the inverse solved in parallel.
static bool dense_inverse_par(std::vector<cplx>& S, int n, cplx* out) {
  unsigned hw = std::thread::hardware_concurrency();
  const int nt = (int)std::max(1u, std::min(hw == 0 ? 4u : hw, 64u));
  std::vector<int> piv(n);
  Team team(nt);
  std::atomic<bool> fail(false);
  cplx inv_piv = 0.0;
  auto worker = [&](int t) {
    for (int k = 0; k < n; ++k) {
      if (t == 0) {
        int pr = k;
        double best = std::abs(S[(size_t)k * n + k]);
        for (int r = k + 1; r < n; ++r) {
          const double v = std::abs(S[(size_t)r * n + k]);
          if (v > best) { best = v; pr = r; }
        }
        piv[k] = pr;
        if (best == 0.0) {
          fail.store(true);
        } else {
          // interchange the trailing columns only: the multipliers of earlier steps
          // stay in place, the convention band_solve applies (as LAPACK's gbtrf)
          if (pr != k)
            for (int c = k; c < n; ++c) std::swap(S[(size_t)k * n + c], S[(size_t)pr * n + c]);
          inv_piv = 1.0 / S[(size_t)k * n + k];
        }
      }
      team.barrier();
      if (fail.load()) return;
      const cplx* rowk = S.data() + (size_t)k * n;
      const cplx ip = inv_piv;
      for (int r = k + 1 + t; r < n; r += nt) {
        cplx* rowr = S.data() + (size_t)r * n;
        const cplx l = rowr[k] * ip;
        rowr[k] = l;
        if (l == 0.0) continue;
        for (int c = k + 1; c < n; ++c) rowr[c] -= l * rowk[c];
      }
      team.barrier();
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker, t);
  worker(0);
  for (auto& th : pool) th.join();
  if (fail.load()) return false;
  parallel_for(n, [&](int c) {
    std::vector<cplx> x(n, cplx(0.0));
    x[c] = 1.0;
    band_solve(S.data(), n, n - 1, n - 1, piv, x.data());
    for (int r = 0; r < n; ++r) out[(size_t)r * n + c] = x[r];
  });
  return true;
}

th_status coarse_setup3(const Geometry& g, const double* k, const double* eps, CoarseBlocks3& cb) {
  const int nc = g.nc, mc = g.mc, q = g.q;
  const int mb = mc * mc;
  const double hc = g.hc;
  cb.mc = mc;
  cb.mb = mb;
  cb.cell.assign((size_t)nc * nc * nc * 4, cplx(0.0));
  cb.rho.assign((size_t)6 * nc * nc, cplx(0.0));
  cb.dn.assign((size_t)mc * mb * 9, cplx(0.0));
  cb.up.assign((size_t)mc * mb * 9, cplx(0.0));
  auto field = [&](int cz, int cy, int cx, const double* f) {
    return f ? f[((size_t)(cz / q) * g.n + cy / q) * g.n + cx / q] : 0.0;
  };
  for (int cz = 0; cz < nc; ++cz)
    for (int cy = 0; cy < nc; ++cy)
      for (int cx = 0; cx < nc; ++cx)
        qsfem27_cell(field(cz, cy, cx, k), field(cz, cy, cx, eps), hc, &cb.cell[(((size_t)cz * nc + cy) * nc + cx) * 4]);
  // face terms: side s = 2 axis + end (axis 0 = x, 1 = y, 2 = z); face cell (f1, f2) over axes (axis+1, axis+2) mod 3
  for (int s = 0; s < 6; ++s) {
    if (!g.robin[s]) continue;
    const int ax = s / 2, end = s % 2;
    const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
    for (int f2 = 0; f2 < nc; ++f2)
      for (int f1 = 0; f1 < nc; ++f1) {
        int c[3];
        c[ax] = end == 0 ? 0 : nc - 1;
        c[a1] = f1;
        c[a2] = f2;
        cb.rho[((size_t)s * nc + f2) * nc + f1] = cplx(0.0, -field(c[2], c[1], c[0], k) * hc * hc);
      }
  }
  // block assembly into the pivot blocks D_z (dense, per slice) and the couplings dn / up
  std::vector<std::vector<cplx>> D(mc);
  for (int j = 0; j < mc; ++j) D[j].assign((size_t)mb * mb, cplx(0.0));
  auto add = [&](cplx v, int za, int ya, int xa, int zb, int yb, int xb) {
    const int a = ya * mc + xa;
    if (za == zb) {
      D[za][(size_t)a * mb + yb * mc + xb] += v;
    } else {
      const int dy = yb - ya + 1, dx = xb - xa + 1;
      if (zb == za + 1) cb.up[((size_t)za * mb + a) * 9 + dy * 3 + dx] += v;
      else cb.dn[((size_t)za * mb + a) * 9 + dy * 3 + dx] += v;
    }
  };
  const double Mq[2][2] = {{1.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 3}};
  for (int cz = 0; cz < nc; ++cz)
    for (int cy = 0; cy < nc; ++cy)
      for (int cx = 0; cx < nc; ++cx) {
        const cplx* dc = &cb.cell[(((size_t)cz * nc + cy) * nc + cx) * 4];
        for (int va = 0; va < 8; ++va)
          for (int vb = 0; vb < 8; ++vb) {
            const int az = va >> 2, ay = (va >> 1) & 1, axx = va & 1;
            const int bz = vb >> 2, by = (vb >> 1) & 1, bx = vb & 1;
            const int nd = (az != bz) + (ay != by) + (axx != bx);
            add(dc[nd], cz + az, cy + ay, cx + axx, cz + bz, cy + by, cx + bx);
          }
      }
  for (int s = 0; s < 6; ++s) {
    if (!g.robin[s]) continue;
    const int ax = s / 2, end = s % 2;
    const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
    for (int f2 = 0; f2 < nc; ++f2)
      for (int f1 = 0; f1 < nc; ++f1) {
        const cplx rv = cb.rho[((size_t)s * nc + f2) * nc + f1];
        for (int i2 = 0; i2 < 2; ++i2)
          for (int i1 = 0; i1 < 2; ++i1)
            for (int j2 = 0; j2 < 2; ++j2)
              for (int j1 = 0; j1 < 2; ++j1) {
                int va[3], vb[3];
                va[ax] = vb[ax] = end == 0 ? 0 : nc;
                va[a1] = f1 + i1;
                va[a2] = f2 + i2;
                vb[a1] = f1 + j1;
                vb[a2] = f2 + j2;
                add(rv * (Mq[i1][j1] * Mq[i2][j2]), va[2], va[1], va[0], vb[2], vb[1], vb[0]);
              }
      }
  }
  // block LU: S_0 = D_0, S_j = D_j - C_{j-1}^T G_{j-1} C_{j-1}, G_j = S_j^{-1},
  // with C_{j-1}[a][b] = A[(j-1, a), (j, b)] = up_{j-1}[a][b - a]
  cb.G.assign((size_t)mc * mb * mb, cplx(0.0));
  std::vector<cplx> T((size_t)mb * mb);
  for (int j = 0; j < mc; ++j) {
    std::vector<cplx>& S = D[j];
    if (j > 0) {
      const cplx* Gp = &cb.G[(size_t)(j - 1) * mb * mb];
      const cplx* Up = &cb.up[(size_t)(j - 1) * mb * 9];
      // T = G_{j-1} C_{j-1}
      parallel_for(mb, [&](int a) {
        cplx* Ta = &T[(size_t)a * mb];
        std::fill(Ta, Ta + mb, cplx(0.0));
        const cplx* Ga = Gp + (size_t)a * mb;
        for (int ap = 0; ap < mb; ++ap) {
          const cplx gv = Ga[ap];
          if (gv == 0.0) continue;
          const int y = ap / mc, x = ap % mc;
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int yb = y + dy, xb = x + dx;
              if (yb < 0 || yb >= mc || xb < 0 || xb >= mc) continue;
              Ta[yb * mc + xb] += gv * Up[(size_t)ap * 9 + (dy + 1) * 3 + (dx + 1)];
            }
        }
      });
      // S -= C^T T: (C^T T)[b][b'] = sum_a C[a][b] T[a][b']
      parallel_for(mb, [&](int b) {
        const int y = b / mc, x = b % mc;
        cplx* Sb = &S[(size_t)b * mb];
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int ya = y - dy, xa = x - dx;  // a with b - a = (dy, dx)
            if (ya < 0 || ya >= mc || xa < 0 || xa >= mc) continue;
            const int a = ya * mc + xa;
            const cplx c = Up[(size_t)a * 9 + (dy + 1) * 3 + (dx + 1)];
            if (c == 0.0) continue;
            const cplx* Ta = &T[(size_t)a * mb];
            for (int bp = 0; bp < mb; ++bp) Sb[bp] -= c * Ta[bp];
          }
      });
    }
    if (!dense_inverse_par(S, mb, &cb.G[(size_t)j * mb * mb])) return TH_ERR_SINGULAR;
    std::vector<cplx>().swap(S);
  }
  return TH_OK;
}

int coarse_chunks(int mc) {
  int P = (int)std::lround(std::sqrt((double)mc));
  P = std::max(1, std::min(P, (mc + 1) / 2));
  return P;
}

th_status coarse_partition(const Geometry& g, const CoarseBlocks& cb, int P, CoarsePart& cp) {
  const int mc = g.mc;
  const size_t mm = (size_t)mc * mc;
  if (P < 1 || 2 * P - 1 > mc) return TH_ERR_ARG;
  cp.P = P;
  cp.mcp = mc + (mc & 1);
  const int ld = cp.mcp;
  // chunk sizes as equal as possible, P - 1 separator rows between them
  const int rows = mc - (P - 1);
  const int base = rows / P, rem = rows % P;
  cp.ca.assign(P, 0);
  cp.cb.assign(P, 0);
  cp.sep.assign(std::max(P - 1, 0), 0);
  int r0 = 0;
  for (int c = 0; c < P; ++c) {
    const int L = base + (c < rem ? 1 : 0);
    cp.ca[c] = r0;
    cp.cb[c] = r0 + L - 1;
    if (c < P - 1) cp.sep[c] = r0 + L;
    r0 += L + 1;
  }
  cp.G.assign((size_t)mc * mc * ld, cplx(0.0));
  cp.LR.assign((size_t)mc * mc * 2 * ld, cplx(0.0));
  const cplx* cl = cb.cl.data();
  const cplx* cd = cb.cd.data();
  const cplx* cu = cb.cu.data();
  std::vector<Mat> Rend(P), Lend(P), Lbeg(P), Rbeg(P);  // spikes at the chunk ends
  std::atomic<int> err(0);
  parallel_for(P, [&](int c) {
    const int a = cp.ca[c], b = cp.cb[c], L = b - a + 1;
    std::vector<Mat> G(L, Mat(mm));
    Mat S(mm), T(mm), U(mm);
    for (int jj = 0; jj < L; ++jj) {
      const int j = a + jj;
      std::fill(S.begin(), S.end(), cplx(0.0));
      const size_t o = (size_t)j * mc;
      for (int r = 0; r < mc; ++r) {
        if (r > 0) S[(size_t)r * mc + r - 1] = cb.dl[o + r];
        S[(size_t)r * mc + r] = cb.dd[o + r];
        if (r + 1 < mc) S[(size_t)r * mc + r + 1] = cb.du[o + r];
      }
      if (jj > 0) {
        const size_t op = (size_t)(j - 1) * mc;
        tri_C_right(mc, cl + op, cd + op, cu + op, G[jj - 1].data(), T.data());  // T = G_{j-1} C_{j-1}
        tri_CT_left(mc, cl + op, cd + op, cu + op, T.data(), U.data());  // B_j T
        for (size_t i = 0; i < mm; ++i) S[i] -= U[i];
      }
      if (!zinverse_serial(mc, S, G[jj].data())) { err.store(1); return; }
      store_padded(mc, ld, G[jj].data(), &cp.G[(size_t)j * mc * ld]);
    }
    // right spike: R_b = G_b C_b, R_j = -G_j C_j R_{j+1}
    if (c < P - 1) {
      Mat R(mm), Rn(mm);
      const size_t ob = (size_t)b * mc;
      tri_C_right(mc, cl + ob, cd + ob, cu + ob, G[L - 1].data(), R.data());
      for (int jj = L - 1; jj >= 0; --jj) {
        const int j = a + jj;
        if (jj < L - 1) {
          const size_t o = (size_t)j * mc;
          tri_C_left(mc, cl + o, cd + o, cu + o, R.data(), T.data());
          zgemm(mc, G[jj].data(), T.data(), Rn.data(), -1.0, false);
          std::swap(R, Rn);
        }
        for (int r = 0; r < mc; ++r)
          std::copy(&R[(size_t)r * mc], &R[(size_t)(r + 1) * mc], &cp.LR[((size_t)j * mc + r) * 2 * ld + ld]);
        if (jj == L - 1) Rend[c] = R;
        if (jj == 0) Rbeg[c] = R;
      }
    }
    // left spike: Z_a = G_a B_a, Z_j = -G_j B_j Z_{j-1}; L_b = Z_b, L_j = Z_j - G_j C_j L_{j+1}
    if (c > 0) {
      std::vector<Mat> Z(L, Mat(mm));
      const size_t oa = (size_t)(a - 1) * mc;  // B_a = C_{a-1}^T
      tri_CT_right(mc, cl + oa, cd + oa, cu + oa, G[0].data(), Z[0].data());
      for (int jj = 1; jj < L; ++jj) {
        const size_t op = (size_t)(a + jj - 1) * mc;
        tri_CT_left(mc, cl + op, cd + op, cu + op, Z[jj - 1].data(), T.data());
        zgemm(mc, G[jj].data(), T.data(), Z[jj].data(), -1.0, false);
      }
      Mat Lc = Z[L - 1];
      for (int jj = L - 1; jj >= 0; --jj) {
        const int j = a + jj;
        if (jj < L - 1) {
          const size_t o = (size_t)j * mc;
          tri_C_left(mc, cl + o, cd + o, cu + o, Lc.data(), T.data());
          Lc = Z[jj];
          zgemm(mc, G[jj].data(), T.data(), Lc.data(), -1.0, true);
        }
        for (int r = 0; r < mc; ++r)
          std::copy(&Lc[(size_t)r * mc], &Lc[(size_t)(r + 1) * mc], &cp.LR[((size_t)j * mc + r) * 2 * ld]);
        if (jj == L - 1) Lend[c] = Lc;
        if (jj == 0) Lbeg[c] = Lc;
      }
    }
  });
  if (err.load()) return TH_ERR_SINGULAR;
  // reduced system on the separators
  const int K = P - 1;
  cp.Gh.assign((size_t)std::max(K, 0) * mc * ld, cplx(0.0));
  cp.Fh.assign((size_t)std::max(K, 0) * mc * ld, cplx(0.0));
  cp.Hh.assign((size_t)std::max(K, 0) * mc * ld, cplx(0.0));
  Mat Ghp(mm), Eprev(mm), S(mm), T(mm), U(mm), W(mm), E(mm), Gk(mm);
  for (int k = 0; k < K; ++k) {
    const int s = cp.sep[k];
    const size_t os = (size_t)s * mc, op = (size_t)(s - 1) * mc;
    std::fill(S.begin(), S.end(), cplx(0.0));
    for (int r = 0; r < mc; ++r) {
      if (r > 0) S[(size_t)r * mc + r - 1] = cb.dl[os + r];
      S[(size_t)r * mc + r] = cb.dd[os + r];
      if (r + 1 < mc) S[(size_t)r * mc + r + 1] = cb.du[os + r];
    }
    // - B_s R^{(k)}_{s-1} - C_s L^{(k+1)}_{s+1}
    tri_CT_left(mc, cl + op, cd + op, cu + op, Rend[k].data(), T.data());
    tri_C_left(mc, cl + os, cd + os, cu + os, Lbeg[k + 1].data(), U.data());
    for (size_t i = 0; i < mm; ++i) S[i] -= T[i] + U[i];
    // What_k = -B_s L^{(k)}_{s-1},  Ehat_k = -C_s R^{(k+1)}_{s+1}
    if (k > 0) {
      tri_CT_left(mc, cl + op, cd + op, cu + op, Lend[k].data(), W.data());
      for (auto& v : W) v = -v;
      // S -= What_k Ghat_{k-1} Ehat_{k-1}
      zgemm_par(mc, Ghp.data(), Eprev.data(), T.data(), 1.0, false);
      zgemm_par(mc, W.data(), T.data(), S.data(), -1.0, true);
    }
    if (!dense_inverse(S, mc, Gk.data())) return TH_ERR_SINGULAR;
    store_padded(mc, ld, Gk.data(), &cp.Gh[(size_t)k * mc * ld]);
    if (k > 0) {
      zgemm_par(mc, Gk.data(), W.data(), T.data(), 1.0, false);
      store_padded(mc, ld, T.data(), &cp.Fh[(size_t)k * mc * ld]);
    }
    if (k < K - 1) {
      tri_C_left(mc, cl + os, cd + os, cu + os, Rbeg[k + 1].data(), E.data());
      for (auto& v : E) v = -v;
      zgemm_par(mc, Gk.data(), E.data(), T.data(), 1.0, false);
      store_padded(mc, ld, T.data(), &cp.Hh[(size_t)k * mc * ld]);
      Eprev = E;
    }
    Ghp = Gk;
  }
  // explicit inverse of the reduced system, one column per unit right-hand side
  // through its block factorisation (forward zhat_k = Ghat_k rhat_k - F_k zhat_{k-1},
  // backward xhat_k = zhat_k - H_k xhat_{k+1}); tasks of up to CB columns of one
  // separator block share each matrix row they read (every column's sums keep
  // their order), tasks in parallel
  if (K > 0) {
    const size_t nred = (size_t)K * mc;
    cp.Sinv.assign(nred * nred, cplx(0.0));
    constexpr int CB = 16;
    const int per_block = (mc + CB - 1) / CB;
    parallel_for(K * per_block, [&](int task) {
      const int k0 = task / per_block, e_begin = (task - k0 * per_block) * CB;
      const int nb = std::min(CB, mc - e_begin);
      std::vector<cplx> z((size_t)CB * nred, cplx(0.0)), xh((size_t)CB * nred, cplx(0.0));  // [column][nred]
      cplx acc[CB];
      for (int k = k0; k < K; ++k) {
        for (int r = 0; r < mc; ++r) {
          if (k == k0) {
            for (int j = 0; j < nb; ++j) z[(size_t)j * nred + (size_t)k * mc + r] = cp.Gh[((size_t)k * mc + r) * ld + e_begin + j];
            continue;
          }
          const cplx* f = &cp.Fh[((size_t)k * mc + r) * ld];
          for (int j = 0; j < nb; ++j) acc[j] = 0.0;
          for (int c2 = 0; c2 < mc; ++c2) {
            const cplx fv = f[c2];
            for (int j = 0; j < nb; ++j) acc[j] += fv * z[(size_t)j * nred + (size_t)(k - 1) * mc + c2];
          }
          for (int j = 0; j < nb; ++j) z[(size_t)j * nred + (size_t)k * mc + r] = -acc[j];
        }
      }
      for (int j = 0; j < nb; ++j)
        for (int r = 0; r < mc; ++r)
          xh[(size_t)j * nred + (size_t)(K - 1) * mc + r] = z[(size_t)j * nred + (size_t)(K - 1) * mc + r];
      for (int k = K - 2; k >= 0; --k) {
        for (int r = 0; r < mc; ++r) {
          const cplx* hrow = &cp.Hh[((size_t)k * mc + r) * ld];
          for (int j = 0; j < nb; ++j) acc[j] = 0.0;
          for (int c2 = 0; c2 < mc; ++c2) {
            const cplx hv = hrow[c2];
            for (int j = 0; j < nb; ++j) acc[j] += hv * xh[(size_t)j * nred + (size_t)(k + 1) * mc + c2];
          }
          for (int j = 0; j < nb; ++j)
            xh[(size_t)j * nred + (size_t)k * mc + r] = z[(size_t)j * nred + (size_t)k * mc + r] - acc[j];
        }
      }
      for (size_t r = 0; r < nred; ++r)
        for (int j = 0; j < nb; ++j) cp.Sinv[r * nred + (size_t)k0 * mc + e_begin + j] = xh[(size_t)j * nred + r];
    });
  }
  return TH_OK;
}

}  // namespace th

namespace th {
// ------------------------------------------------ Galerkin p-type coarsening
// Section 4 ("Standard Galerkin p-type coarsening"): the coarse space is Q_q,
// q = p/2, on the same mesh, in the nodal basis of the equispaced points of
// each cell (the coarse-grid vertices, the basis the prolongation I_P of
// Section 4.2 interpolates from), so I_P is the embedding and the coarse matrix
// is the fine form restricted to Q_q.  With constant coefficients per cell and
// exact integration this is, per cell e,
//   Kq (x) Mq + Mq (x) Kq - (k_e^2 (1 + i alpha_c) + i eps_e) h^2 Mq (x) Mq
// plus -i k_e h Mq on each Robin edge, Kq / Mq the 1-D stiffness / mass of the
// degree-q equispaced Lagrange basis on [0, 1].
th_status galerkin_setup(const Geometry& g, const double* k, const double* eps, double alpha_c, GalBlocks& gb) {
  if (g.dim != 2) return TH_ERR_UNSUPPORTED;
  const int q = g.q, mc = g.mc, n = g.n, S = 2 * q + 1, nq1 = q + 1;
  gb.q = q;
  gb.mc = mc;
  gb.nblk = n;
  // 1-D equispaced reference matrices, Gauss rule exact for degree 2q
  std::vector<double> eq(nq1), xq, wq;
  for (int b = 0; b <= q; ++b) eq[b] = (double)b / q;
  gauss_rule(q + 2, xq, wq);
  std::vector<double> Mq(nq1 * nq1, 0.0), Kq(nq1 * nq1, 0.0);
  auto dlag = [&](int a, double x) {  // derivative of the a-th equispaced Lagrange polynomial
    double s = 0.0;
    for (int j = 0; j <= q; ++j) {
      if (j == a) continue;
      double t = 1.0 / (eq[a] - eq[j]);
      for (int l = 0; l <= q; ++l)
        if (l != a && l != j) t *= (x - eq[l]) / (eq[a] - eq[l]);
      s += t;
    }
    return s;
  };
  for (int a = 0; a <= q; ++a)
    for (int b = 0; b <= q; ++b)
      for (size_t t = 0; t < xq.size(); ++t) {
        Mq[a * nq1 + b] += wq[t] * lagrange_value(eq, a, xq[t]) * lagrange_value(eq, b, xq[t]);
        Kq[a * nq1 + b] += wq[t] * dlag(a, xq[t]) * dlag(b, xq[t]);
      }
  // stencil: st[(y mc + x) S^2 + (dy + q) S + (dx + q)] = A_c[(y, x), (y + dy, x + dx)]
  gb.st.assign((size_t)mc * mc * S * S, cplx(0.0));
  auto add = [&](int ya, int xa, int yb, int xb, cplx v) {
    gb.st[((size_t)ya * mc + xa) * S * S + (size_t)(yb - ya + q) * S + (xb - xa + q)] += v;
  };
  const double h = g.h;
  for (int cy = 0; cy < n; ++cy)
    for (int cx = 0; cx < n; ++cx) {
      const size_t f = (size_t)cy * n + cx;
      const double kk = k[f], ee = eps ? eps[f] : 0.0;
      const cplx cvol(kk * kk, alpha_c * kk * kk + ee);
      for (int ay = 0; ay <= q; ++ay)
        for (int ax = 0; ax <= q; ++ax)
          for (int by = 0; by <= q; ++by)
            for (int bx = 0; bx <= q; ++bx) {
              const double mx = Mq[ax * nq1 + bx], my = Mq[ay * nq1 + by];
              const double kx = Kq[ax * nq1 + bx], ky = Kq[ay * nq1 + by];
              const cplx v = cplx(kx * my + mx * ky, 0.0) - cvol * (h * h * mx * my);
              add(cy * q + ay, cx * q + ax, cy * q + by, cx * q + bx, v);
            }
    }
  for (int s = 0; s < 4; ++s) {
    if (!g.robin[s]) continue;
    for (int t = 0; t < n; ++t) {
      // edge cell and the nodes along the edge: side s = 0/1 x lo/hi (nodes vary in y), 2/3 y lo/hi
      const int cx = s < 2 ? (s == 0 ? 0 : n - 1) : t, cy = s < 2 ? t : (s == 2 ? 0 : n - 1);
      const cplx rv(0.0, -k[(size_t)cy * n + cx] * h);
      for (int a = 0; a <= q; ++a)
        for (int b = 0; b <= q; ++b) {
          const cplx v = rv * Mq[a * nq1 + b];
          if (s < 2) {
            const int x = s == 0 ? 0 : mc - 1;
            add(t * q + a, x, t * q + b, x, v);
          } else {
            const int y = s == 2 ? 0 : mc - 1;
            add(y, t * q + a, y, t * q + b, v);
          }
        }
    }
  }
  // block LU over the row groups: G_j = (D_j - L_j G_{j-1} U_{j-1})^{-1}.  Only
  // the last row of group j-1 couples to group j, so only that mc x mc corner of
  // G_{j-1} enters the Schur complement.
  const size_t gtot = (size_t)gal_goff(n, q, mc);
  gb.G.assign(gtot, cplx(0.0));
  for (int j = 0; j < n; ++j) {
    const int lo = gal_row_lo(j, q), hi = gal_row_hi(j, q), Sj = (hi - lo + 1) * mc;
    std::vector<cplx> D((size_t)Sj * Sj, cplx(0.0));
    parallel_for(Sj, [&](int a) {
      const int ya = lo + a / mc, xa = a % mc;
      const cplx* sa = &gb.st[((size_t)ya * mc + xa) * S * S];
      for (int dy = -q; dy <= q; ++dy) {
        const int yb = ya + dy;
        if (yb < lo || yb > hi) continue;
        for (int dx = -q; dx <= q; ++dx) {
          const int xb = xa + dx;
          if (xb < 0 || xb >= mc) continue;
          D[(size_t)a * Sj + (size_t)(yb - lo) * mc + xb] += sa[(dy + q) * S + dx + q];
        }
      }
    });
    if (j > 0) {
      const int plo = gal_row_lo(j - 1, q), Sp = (gal_row_hi(j - 1, q) - plo + 1) * mc;
      const int yl = lo - 1;  // the last row of group j-1
      const cplx* Gp = &gb.G[(size_t)gal_goff(j - 1, q, mc)];
      const size_t c0 = (size_t)Sp - mc;  // local index of (yl, 0) in group j-1
      // T[a][d] = sum_c L[a][c] Gll[c][d], c, d on row yl
      std::vector<cplx> T((size_t)Sj * mc, cplx(0.0));
      parallel_for(Sj, [&](int a) {
        const int ya = lo + a / mc, xa = a % mc, dy = yl - ya;
        if (dy < -q) return;
        const cplx* sa = &gb.st[((size_t)ya * mc + xa) * S * S];
        for (int dx = -q; dx <= q; ++dx) {
          const int xc = xa + dx;
          if (xc < 0 || xc >= mc) continue;
          const cplx l = sa[(dy + q) * S + dx + q];
          if (l == 0.0) continue;
          const cplx* grow = Gp + (c0 + xc) * Sp + c0;
          for (int d = 0; d < mc; ++d) T[(size_t)a * mc + d] += l * grow[d];
        }
      });
      // D[a][b] -= sum_d T[a][d] U[d][b], U[d][b] = A_c[(yl, d), b]
      parallel_for(Sj, [&](int a) {
        for (int d = 0; d < mc; ++d) {
          const cplx t = T[(size_t)a * mc + d];
          if (t == 0.0) continue;
          const cplx* sd = &gb.st[((size_t)yl * mc + d) * S * S];
          for (int dy = 1; dy <= q; ++dy) {
            const int yb = yl + dy;
            if (yb > hi) break;
            for (int dx = -q; dx <= q; ++dx) {
              const int xb = d + dx;
              if (xb < 0 || xb >= mc) continue;
              D[(size_t)a * Sj + (size_t)(yb - lo) * mc + xb] -= t * sd[(dy + q) * S + dx + q];
            }
          }
        }
      });
    }
    if (!dense_inverse_par(D, Sj, &gb.G[(size_t)gal_goff(j, q, mc)])) return TH_ERR_SINGULAR;
  }
  return TH_OK;
}
}  // namespace th
