// Internal declarations of the two-grid Helmholtz library (host + device).
#pragma once

#include "kernels.h"

#include <complex>
#include <cstddef>
#include <cstdint>
#include <functional>
#include <vector>

#include "../../include/th.h"

namespace th {

using cplx = std::complex<double>;

constexpr int kMaxP = 8;

// ---------------------------------------------------------------- host setup
struct Ref1D {
  int p = 0;
  std::vector<double> nodes;  // GLL points on [0,1], p+1
  std::vector<double> M, K;   // (p+1)^2 row-major, exact mass / stiffness
  std::vector<double> Pw;     // (p+1) x (p/2+1): l^eq_b(xi_a), degree-p/2 interpolation
};
Ref1D reference_1d(int p);

struct Block1D {
  std::vector<int> start, size;  // cell ranges of the U blocks along one axis
};
Block1D partition_1d(int n, int l_dd);

// Geometry of the fine mesh, the partition and the coarse mesh.
constexpr int kBox = 12;  // ints per subdomain box

struct Geometry {
  int dim = 2;              // 2 or 3
  int n = 0, p = 0, q = 0;  // cells, order, p/2
  int m = 0;                // fine nodes per direction n p + 1
  long long N = 0;          // fine dofs m^dim
  int nc = 0;               // coarse cells per direction n p / 2
  int mc = 0;               // coarse nodes per direction nc + 1
  long long Nc = 0;         // coarse dofs mc^dim
  double h = 0, hc = 0;
  int robin[6] = {0, 0, 0, 0, 0, 0};  // x lo, x hi, y lo, y hi, z lo, z hi
  int dirichlet[6] = {0, 0, 0, 0, 0, 0};  // sides of Gamma_0 (u = 0), same order (2-D only)
  // partition
  int l_dd = 0;
  Block1D blk;              // same along x and y
  int nb = 0;               // blocks per direction
  int nsub = 0;             // nb^dim
  int Lw = 0, Lu = 0;       // max Omega / U box width in dofs
  int NC = 0, NR = 0;       // Lw^dim columns, Lu^dim rows of an inverse-row block
  // per-subdomain boxes (dof coordinates), kBox ints each:
  // ox, oy, wx, wy, ux, uy, vx, vy, oz, wz, uz, vz (2-D: oz = uz = 0, wz = vz = 1)
  std::vector<int> box;
  // 1-D combine table: per fine 1-D node i: (b0, r0, b1, r1), b1 = -1 if only one block
  std::vector<int> ctab;
  std::vector<int> mult1d;  // multiplicity along one axis (1 or 2)
};
th_status make_geometry(const th_mesh& mesh, const th_params& prm, Geometry& g);

// Dense FP64 inverse rows of subdomain `sub`: NR x NC row-major (zero padded).
th_status subdomain_inverse_rows(const Geometry& g, const Ref1D& ref, const double* k,
                                 const double* eps, double alpha_s, int sub, cplx* out);

// All subdomains, threaded; distinct subdomains with identical data are computed once.
th_status all_inverse_rows(const Geometry& g, const Ref1D& ref, const double* k, const double* eps,
                           double alpha_s, std::vector<cplx>& out);

// QSFEM coarse cell coefficients (d0, d1, d2).
void qsfem_cell(double k, double eps, double hc, cplx d[3]);

// Coarse operator in block-tridiagonal form (rows of the coarse grid) and its
// FP64 block factorisation G_j = S_j^{-1}.
struct CoarseBlocks {
  int mc = 0;
  std::vector<cplx> cell;         // nc^2 x 3 (d0, d1, d2) per coarse cell
  std::vector<cplx> rho[4];       // per side: nc edges, -i k hc (0 for Neumann)
  std::vector<cplx> dl, dd, du;   // D_j tridiagonal, mc x mc
  std::vector<cplx> cl, cd, cu;   // C_j = A[row j, row j+1] tridiagonal, mc x mc (row mc-1 unused)
  std::vector<cplx> G;            // mc blocks of mc x mc
};
// block_inverses = false leaves G empty (only the unpartitioned FP64 sweep of
// th_coarse_solve_noalloc reads it).
th_status coarse_setup(const Geometry& g, const double* k, const double* eps, CoarseBlocks& cb,
                       bool block_inverses = true);

// 3-D coarse operator (fitted 27-point scheme) in z-slice block form: the
// unknowns of slice j are the mb = mc^2 coarse nodes of that slice.
struct CoarseBlocks3 {
  int mc = 0, mb = 0;
  std::vector<cplx> cell;  // nc^3 x 4: d_0..d_3 per coarse cell (pair weight by differing coordinates)
  std::vector<cplx> rho;   // 6 x nc^2: -i k h_c^2 per face cell (0 where Neumann)
  std::vector<cplx> dn;    // mc x mb x 9: A[(j, a), (j-1, a + (dy, dx))], dy, dx in -1..1 (slice 0: unused)
  std::vector<cplx> up;    // mc x mb x 9: A[(j, a), (j+1, a + (dy, dx))] (last slice: unused)
  std::vector<cplx> G;     // mc blocks of mb x mb: inverses of the block-LU pivots
};
void qsfem27_cell(double k, double eps, double hc, cplx d[4]);
th_status coarse_setup3(const Geometry& g, const double* k, const double* eps, CoarseBlocks3& cb);

// Galerkin p-type coarsening (2-D): the coarse operator as a (2q+1)^2-point
// stencil per coarse node, and the FP64 block inverses of its block-tridiagonal
// form over the row groups gal_row_lo(j)..gal_row_hi(j) (kernels.h).
struct GalBlocks {
  int q = 0, mc = 0, nblk = 0;
  std::vector<cplx> st;  // mc^2 x (2q+1)^2
  std::vector<cplx> G;   // block j at gal_goff(j), (rows_j mc)^2 row-major
};
th_status galerkin_setup(const Geometry& g, const double* k, const double* eps, double alpha_c, GalBlocks& gb);

// Partitioned form of the coarse block-tridiagonal system (see coarse_partition).
struct CoarsePart {
  int P = 1;                      // chunks of coarse rows
  int mcp = 0;                    // padded row stride of dense blocks (even)
  std::vector<int> ca, cb;        // chunk row ranges [ca, cb]
  std::vector<int> sep;           // separator rows, P - 1
  std::vector<cplx> G;            // mc blocks (chunk rows; separator slots zero), mc x mcp each
  std::vector<cplx> LR;           // mc blocks of mc x (2 mcp): [L_j | R_j] spikes
  std::vector<cplx> Gh, Fh, Hh;   // P - 1 blocks each, mc x mcp: reduced factors
  std::vector<cplx> Sinv;         // explicit inverse of the reduced system, (P-1) mc square
};
th_status coarse_partition(const Geometry& g, const CoarseBlocks& cb, int P, CoarsePart& cp);
int coarse_chunks(int mc);

// Transfer tables.
struct TransferTables {
  int q = 0, rmax = 0;
  std::vector<int> pj0;        // per fine 1-D node: first coarse node of its cell
  std::vector<double> pw;      // per fine 1-D node: q+1 weights
  std::vector<int> rcnt;       // per coarse 1-D node: count of fine contributors
  std::vector<int> ridx;       // per coarse 1-D node: rmax fine indices
  std::vector<double> rw;      // per coarse 1-D node: rmax weights
};
void transfer_tables(const Geometry& g, const Ref1D& ref, TransferTables& t);

void parallel_for(int n, const std::function<void(int)>& f);

// ---------------------------------------------------------------- device side
struct DevBufs;  // defined in api.cpp

}  // namespace th
