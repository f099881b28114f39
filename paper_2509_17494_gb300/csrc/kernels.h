// Kernel argument blocks and host launchers (device code lives in the .cu files).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace th {

template <typename T> struct Cx;
template <> struct Cx<double> { using t = double2; };
template <> struct Cx<float> { using t = float2; };

// Double-single number: the unevaluated sum h + l of two floats, |l| <= ulp(h) / 2
// (Dekker 1971): 48 significant bits from FP32 arithmetic.  The device
// operators are defined where they are used (fine.cu).  In the mixed form's
// outer residual, global inputs are FP64 (split exactly into h + l on load) and
// the output is FP32.
struct ds {
  float h, l;
  ds() = default;
  __host__ __device__ constexpr ds(float v) : h(v), l(0.f) {}
  __host__ __device__ constexpr ds(int v) : h((float)v), l(0.f) {}
  __host__ __device__ constexpr ds(float a, float b) : h(a), l(b) {}
};
struct cds {
  ds x, y;
};
template <> struct Cx<ds> { using t = cds; };

#if defined(__CUDACC__)
// c + a b as one fused multiply-add.  Accumulations are written as chains of
// these: the compiler may not reassociate acc + (a b + c d) into two FMAs.
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
// acc += a b (complex)
template <typename C>
__device__ __forceinline__ void cmadd(C& acc, C a, C b) {
  acc.x = fmadd(a.x, b.x, acc.x);
  acc.x = fmadd(-a.y, b.y, acc.x);
  acc.y = fmadd(a.x, b.y, acc.y);
  acc.y = fmadd(a.y, b.x, acc.y);
}
#endif
inline ds ds_from_host(double v) {
  const float h = (float)v;
  return ds(h, (float)(v - (double)h));
}

// ---------------------------------------------------------------- K1 fine apply
template <typename T>
struct FineArgs {
  const typename Cx<T>::t* u;
  const typename Cx<T>::t* f;  // used when residual != 0
  typename Cx<T>::t* y;
  const T* kc;                 // k per cell
  const T* ec;                 // eps per cell
  long long N;                 // stride between right-hand sides
  int n, m, p;
  int robin;                   // bit s set = side s absorbing (x lo, x hi, y lo, y hi)
  int dirichlet;               // bit s set = side s on Gamma_0: identity rows and columns there
  int residual;                // 0: y = OP u;  1: y = f - OP u
  int out64;                   // double-single apply only: y in FP64 (the rounded sum of each pair) instead of FP32
  int tc;                      // tile edge in cells (0: default for p)
  T h, h2, alpha;              // alpha = shift (0 for A)
  T M[81], K[81];              // 1-D reference mass / stiffness, (p+1)^2
  // even / odd halves (both matrices are centrosymmetric), H = p/2, 1/2 folded in:
  // ME[a][b] = (M[a][b] + M[a][p-b]) / 2 (b < H), ME[a][H] = M[a][H]; MO[a][b] = (M[a][b] - M[a][p-b]) / 2
  T ME[25], MO[16], KE[25], KO[16];
  // Where the operand comes from (FP32 / FP64 forms only; the fused cycle):
  //   src 0: u;
  //   src 1: the RAS-like average of the subdomain results, u_j = sum of the
  //          V entries of the U boxes that hold node j (the weights 1/L_j are
  //          in the rows), in the order of k_dd_combine;
  //   src 2: uin + omega I_P uc (the prolonged coarse correction), in the
  //          order of k_prolong.
  // With src != 0 the operand at the owned nodes is also written to uout
  // (which must not alias uin).
  int src;
  const typename Cx<T>::t* V;  // src 1: [rhs][nsub][NR]
  const int4* ctab;            // src 1: per 1-D node (b0, r0, b1, r1)
  int nb, Lu, NR, nsub;
  const typename Cx<T>::t* uin;  // src 2
  const typename Cx<T>::t* uc;   // src 2: coarse correction, [rhs][Nc]
  const int* pj0;                // src 2: per fine 1-D node, first coarse node of its cell
  const T* pw;                   // src 2: per fine 1-D node, q + 1 weights
  long long Nc;
  int mc, q;
  T omega;
  typename Cx<T>::t* uout;
};
template <typename T>
cudaError_t launch_fine_apply(const FineArgs<T>& a, int nrhs, cudaStream_t s);

// ------------------------------------------------------- K3 DD block apply
enum WKind { W_FP64 = 0, W_FP32 = 1, W_BF16 = 2, W_FP16 = 3 };
template <typename T>
struct DDArgs {
  const typename Cx<T>::t* r;   // residual, [rhs][N]
  typename Cx<T>::t* V;         // per-subdomain results, [rhs][nsub][NR]
  const void* W;                // inverse rows, [sub][chunk][NR] 16-byte chunks
  const int* box;               // kBox = 12 ints per subdomain (see th_internal.h)
  const float* wscale;          // per-subdomain scale (FP16 rows), or null
  long long N;
  int nsub, m, Lw, NC, NCH, NR, G, nrhs;
  int stream_v2;                // launch_dd_stream: 1 = producer-warp variant (k_dd_stream2)
  int stream_small;             // launch_dd_stream (k_dd_stream): 1 = 20 KB ring stages, three CTAs per SM
  int stream_pk;                // launch_dd_stream (k_dd_stream, FP32 on BF16/FP16 rows): paired FP32 FMAs
};
template <typename T>
cudaError_t launch_dd_apply(const DDArgs<T>& a, int kind, int grid_cap, cudaStream_t s);
// TMA-streamed variant (persistent, one CTA per SM); *err is set to 1 if a bounded wait gave up
template <typename T>
cudaError_t launch_dd_stream(const DDArgs<T>& a, int kind, int* err, int sms, cudaStream_t s);

// ------------------------------------------------------- K3b batched DD on tensor cores
// V[rhs][sub][row] = W_sub X_sub for a tile of NB right-hand sides with
// tcgen05.mma (BF16 operands, FP32 accumulators in tensor memory).
struct DDUmmaArgs {
  const float2* r;        // residual, [rhs][N], FP32 complex
  float2* V;              // [rhs][nsub][NR]
  const unsigned char* W; // BF16 rows in the UMMA core-matrix layout (see setup)
  const int* box;         // 12 ints per subdomain
  int* err;               // set to 1 when a bounded wait gives up
  long long N;
  int nsub, m, Lw, NC, NR, nrhs;
  int M8, K8;             // row and column core-matrix counts (rows <= 128, K8 even)
  int dim3;               // 1: 3-D boxes (z origin and width used by the gather)
};
cudaError_t launch_dd_umma(const DDUmmaArgs& a, int sms, cudaStream_t s);
size_t dd_umma_bytes_per_sub(int NR, int NC);

// ------------------------------------------------------- K4 DD combine
template <typename T>
struct CombineArgs {
  const typename Cx<T>::t* V;   // [rhs][nsub][NR]
  typename Cx<T>::t* u;         // [rhs][N]
  const int4* ctab;             // per 1-D node: (b0, r0, b1, r1)
  long long N;
  int m, nb, Lu, NR, nsub, accumulate;
  // fused cycle: with uin set the result is uin + average (u is not read);
  // with wide set it goes, widened to FP64, to wide (added to it if
  // wide_acc) instead of u
  const typename Cx<T>::t* uin;
  double2* wide;
  int wide_acc;
};
template <typename T>
cudaError_t launch_dd_combine(const CombineArgs<T>& a, int nrhs, cudaStream_t s);

// coarse node (ix, iy) of an mc x mc grid on a side of Gamma_0 (bits: x lo, x hi, y lo, y hi)
__host__ __device__ inline bool coarse_on_gamma0(int bits, int ix, int iy, int mc) {
  return ((bits & 1) && ix == 0) || ((bits & 2) && ix == mc - 1) || ((bits & 4) && iy == 0) ||
         ((bits & 8) && iy == mc - 1);
}

// ------------------------------------------------------- K5/K6 transfers
template <typename T>
struct TransferArgs {
  const typename Cx<T>::t* in;
  typename Cx<T>::t* out;
  const int* pj0;  const T* pw;                        // prolongation tables (per fine 1-D node)
  const int* ridx; const T* rw; int rmax;              // restriction tables (per coarse 1-D node)
  long long N, Nc;
  int m, mc, q;
  T omega;
  int dirichlet;               // restriction: bit s set = coarse nodes of side s get 0 (x lo, x hi, y lo, y hi)
};
template <typename T>
cudaError_t launch_restrict(const TransferArgs<T>& a, int nrhs, cudaStream_t s);
template <typename T>
cudaError_t launch_prolong(const TransferArgs<T>& a, int nrhs, cudaStream_t s);

// ------------------------------------------------------- K7 coarse apply
template <typename T>
struct CoarseApplyArgs {
  const typename Cx<T>::t* x;
  typename Cx<T>::t* y;
  const typename Cx<T>::t* cell;   // nc^2 x 3 (d0, d1, d2)
  const typename Cx<T>::t* rho;    // 4 x nc (per side), zero where Neumann
  long long Nc;
  int nc, mc;
  int dirichlet;                   // bit s set = side s on Gamma_0: identity rows, zero columns
  const typename Cx<T>::t* f;      // non-null: y = f - A_q x (the residual) instead of A_q x
};
template <typename T>
cudaError_t launch_coarse_apply(const CoarseApplyArgs<T>& a, int nrhs, cudaStream_t s);
// u += w, n complex FP32 entries
cudaError_t launch_cadd32(float2* u, const float2* w, long long n, cudaStream_t s);

// ------------------------------------------------------- K8 coarse solve
template <typename T>
struct CoarseSolveArgs {
  const typename Cx<T>::t* rhs;    // [rhs][Nc]
  typename Cx<T>::t* x;            // [rhs][Nc]
  typename Cx<T>::t* z;            // scratch [rhs][Nc]
  const typename Cx<T>::t* G;      // mc blocks of mc x mc
  const typename Cx<T>::t* cl;     // C_j diagonals, mc x mc
  const typename Cx<T>::t* cd;
  const typename Cx<T>::t* cu;
  long long Nc;
  int mc, rpc;                     // rows per CTA
};
template <typename T>
cudaError_t launch_coarse_solve(const CoarseSolveArgs<T>& a, int nrhs, int cluster, cudaStream_t s);

// ------------------------------------------------------- K8 partitioned coarse solve
template <typename T>
struct CoarsePartArgs {
  const typename Cx<T>::t* b;    // [rhs][Nc]
  typename Cx<T>::t* x;          // [rhs][Nc]
  const typename Cx<T>::t* G;    // chunk-row block inverses, mc blocks of mc x mcp
  const typename Cx<T>::t* LR;   // spikes [L_j | R_j], mc blocks of mc x 2 mcp
  const typename Cx<T>::t* Sinv; // explicit inverse of the reduced separator system, nred x ldS
  typename Cx<T>::t* rhat;       // scratch: reduced right-hand sides, [rhs][nred]
  const typename Cx<T>::t* cl;   // C_j diagonals
  const typename Cx<T>::t* cd;
  const typename Cx<T>::t* cu;
  const int* ca;                 // chunk first rows
  const int* cb;                 // chunk last rows
  const int* sep;                // separator rows
  const int* chunk_of;           // per row: chunk index, or -1 for a separator
  // multi-right-hand-side sweep: G_j transposed, [j][column][mcr] (rows padded to mcr = cluster * rpcm)
  const typename Cx<T>::t* Gt;
  // spikes transposed, [j][col][mcr] (col < 2 mcp), for the grouped spike correction; or null
  const typename Cx<T>::t* LRt;
  long long Nc;
  int mc, mcp, P, rpc, Lmax, nred;
  int mcr, rpcm, nrhs;           // rpcm: rows per CTA of the multi-rhs sweep (even)
  int ldS;                       // row stride of Sinv (nred rounded up to even)
  int sweep_variant;             // one-rhs chunk sweep: 0 two-phase (512 threads), 1 one barrier per step (1024),
                                 // 2 st.async row exchange on mbarriers (no cluster barrier per step)
  int* err;                      // device flag set by a bounded wait that gave up (variant 2)
  int multi_variant;             // 8 or more right-hand sides: 0 per-tile cluster sweep, 1 column groups per CTA,
                                 // 2 column groups + tensor-core separator and spike products (umma below)
  int nsm;                       // SMs of the device (column groups are sized to fill them in one wave)
  // reduced right-hand sides as split-BF16 operand chunks (tensor-core path), else null:
  // [rhs / 64][nkc_s][re hi | im hi | re lo | im lo][umma_off32(rhs % 64, k % 32)]
  unsigned char* rst;
  int nkc_s;
  const struct CoarseUmmaArgs* umma;  // host-side description of the tensor-core products, or null
  // one right-hand side (FP32): the upper-triangle 64 x 64 blocks of the complex-symmetric Sinv
  // (row-major, zero padded), their (I, J) tile pairs, and the partial products [T][T][64]; or null
  const typename Cx<T>::t* Ssym;
  const int2* sym_ij;
  typename Cx<T>::t* spart;
  int Tsym, nsym;
};
template <typename T>
cudaError_t launch_coarse_part(const CoarsePartArgs<T>& a, int nrhs, int cluster, cudaStream_t s);

// Offset (in elements) of entry (r, k) of a 32-column chunk in the tensor
// cores' no-swizzle K-major operand layout: core matrices of 8 rows x 8
// 16-bit entries (128 bytes), arranged [r / 8][k / 8] with k / 8 fastest.
__host__ __device__ inline int umma_off32(int r, int k) {
  return (((r >> 3) * 4 + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

// K8c: one 128-row tile of a tensor-core coarse product (coarse_umma.cu)
struct CoarseTile {
  long long a_off;  // byte offset of the tile's A chunks (nkc x 32 KB)
  int nkc;          // chunks of 32 columns
  int row0;         // separator product: first reduced index; spikes: x index of the first row
  int rows;         // valid rows (<= 128)
  int b0, b1;       // spikes: separator of the first and second column block (b1 = -1: one block);
                    // separator product split over K: first chunk and split index
};
struct CoarseUmmaArgs {
  const unsigned char* As;  // split-BF16 reduced inverse, ntiles_s tiles
  const unsigned char* Al;  // split-BF16 spikes, ntiles_l tiles
  const CoarseTile* tiles_s;
  const CoarseTile* tiles_l;
  int ntiles_s, ntiles_l;
  const unsigned char* rst;  // reduced right-hand sides, 16 KB chunks [rhs / 64][nkc_s]
  unsigned char* xst;        // separator values, 16 KB chunks [rhs / 64][nsep][nkc_m] (written by MODE 0)
  float2* x;                 // [rhs][Nc]
  const int* sep;            // separator rows
  long long Nc;
  int mc, nsep, nkc_s, nkc_m, nrhs;
  int* err;
  // MODE 0 split over K (nsplit > 1): tile entries carry their first chunk (b0) and split
  // index (b1); partial products go to spart [nsplit][nrhs_cap][nred] and k_sep_split_sum
  // adds them in a fixed order
  float2* spart;
  int nsplit, nrhs_cap, nred;
};
cudaError_t launch_coarse_umma(const CoarseUmmaArgs& a, int mode, int sms, cudaStream_t s);

// ------------------------------------------------------- 3-D (unit cube, Q2)
template <typename T>
struct Fine3Args {
  const typename Cx<T>::t* u;
  const typename Cx<T>::t* f;  // used when residual != 0
  typename Cx<T>::t* y;
  typename Cx<T>::t* ycell;    // scratch [rhs][n^3][32]: per-cell local outputs
  const T* kc;                 // k per cell
  const T* ec;                 // eps per cell
  long long N, ncell;          // m^3, n^3
  int n, m;
  int robin;                   // bit s = side s absorbing (x lo, x hi, y lo, y hi, z lo, z hi)
  int residual;
  T h, alpha;
  T M[9], K[9];                // 1-D reference mass / stiffness (p = 2)
};
template <typename T>
cudaError_t launch_fine3(const Fine3Args<T>& a, int nrhs, cudaStream_t s);
template <typename T>
cudaError_t launch_dd_combine3(const CombineArgs<T>& a, int nrhs, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict3(const TransferArgs<T>& a, int nrhs, cudaStream_t s);
template <typename T>
cudaError_t launch_prolong3(const TransferArgs<T>& a, int nrhs, cudaStream_t s);
// (CoarseApplyArgs: cell = nc^3 x 4 pair weights, rho = 6 x nc^2 face terms)
template <typename T>
cudaError_t launch_coarse_apply3(const CoarseApplyArgs<T>& a, int nrhs, cudaStream_t s);
template <typename T>
struct Sweep3Args {
  const typename Cx<T>::t* b;    // [rhs][Nc]
  typename Cx<T>::t* x;          // [rhs][Nc]
  typename Cx<T>::t* t;          // scratch [rhs][mb]
  const typename Cx<T>::t* G;    // mc blocks of mb x mb
  const typename Cx<T>::t* dn;   // mc x mb x 9 couplings to the slice below
  const typename Cx<T>::t* up;   // mc x mb x 9 couplings to the slice above
  long long Nc;
  int mc, mb, nrhs;
};
template <typename T>
cudaError_t launch_sweep3(const Sweep3Args<T>& a, cudaStream_t s);

// ------------------------------------------ Galerkin p-type coarsening (2-D)
// Row groups of the coarse node grid: [0, q], then [j q + 1, (j + 1) q] for
// j = 1 .. n - 1, so that only the last row of group j couples to group j + 1.
__host__ __device__ inline int gal_row_lo(int j, int q) { return j == 0 ? 0 : j * q + 1; }
__host__ __device__ inline int gal_row_hi(int j, int q) { return (j + 1) * q; }
__host__ __device__ inline int gal_group(int row, int q) { return row <= q ? 0 : (row - 1) / q; }
// offset of block j in the concatenated inverses (block 0: ((q+1) mc)^2, the rest (q mc)^2)
__host__ __device__ inline long long gal_goff(int j, int q, int mc) {
  const long long s0 = (long long)(q + 1) * mc, s = (long long)q * mc;
  return j == 0 ? 0 : s0 * s0 + (long long)(j - 1) * s * s;
}
template <typename T>
struct GalArgs {
  const typename Cx<T>::t* st;  // mc^2 x (2q+1)^2 stencil
  const typename Cx<T>::t* G;   // block inverses
  const typename Cx<T>::t* b;   // [rhs][Nc]
  typename Cx<T>::t* x;         // [rhs][Nc]
  long long Nc;
  int q, mc, nblk, nrhs;
};
// y = A_c x (x = a.b, y = a.x)
template <typename T>
cudaError_t launch_gal_apply(const GalArgs<T>& a, cudaStream_t s);
// x = A_c^{-1} b: block forward and backward sweeps, one launch per block step
template <typename T>
cudaError_t launch_gal_solve(const GalArgs<T>& a, cudaStream_t s);
int gal_solve_launches(int nblk);

// ------------------------------------------------------- vectors (K9/K10)
cudaError_t launch_d2f(const double* in, float* out, long long n, cudaStream_t s);
cudaError_t launch_f2d(const float* in, double* out, long long n, int accumulate, cudaStream_t s);
// y[r] = a * x[r] + b * y[r] (complex a per rhs from device array, b real); generic axpby on complex vectors
cudaError_t launch_zaxpy_f64(const double2* x, double2* y, double alpha, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_zaxpy(const typename Cx<T>::t* x, typename Cx<T>::t* y, T alpha, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_zero(typename Cx<T>::t* x, long long n, cudaStream_t s);

// multi-dot: h[rhs][i] = sum_n conj(V_i[rhs][n]) w[rhs][n], i = 0..nv-1, V_i at Vbase + i*vstride;
// self = 1 appends h[rhs][nv] = ||w[rhs]||^2 (row stride nv + self).  Partial sums in `part`
// ([rhs][nv + self][nblk]) then a fixed-order reduction.
int mdot_blocks(long long N);
cudaError_t launch_mdot(const double2* Vbase, long long vstride, const double2* w, long long N,
                        int nv, int self, int nrhs, double2* part, double2* h, int nblk, cudaStream_t s);
// w[rhs] -= sum_i h[rhs][i] V_i[rhs]  (sign = -1) or += (sign = +1)
cudaError_t launch_maxpy(const double2* Vbase, long long vstride, const double2* h, int hstride,
                         double2* w, long long N, int nv, int nrhs, double sign, cudaStream_t s);
// nrm2[rhs] = ||w[rhs]||^2 (fixed-order two-pass reduction into part/out)
cudaError_t launch_norm2(const double2* w, long long N, int nrhs, double* part, double* out,
                         int nblk, cudaStream_t s);
// the same three in double-single arithmetic (the mixed form's FGMRES; vec.cu)
// split != 0: the basis vectors V_i stored as (re h, re l, im h, im l) floats (launch_scale_split)
cudaError_t launch_mdot_ds(const double2* Vbase, long long vstride, const double2* w, long long N, int nv, int self,
                           int nrhs, double2* part, double2* h, int nblk, int split, cudaStream_t s);
cudaError_t launch_maxpy_ds(const double2* Vbase, long long vstride, const double2* h, int hstride, double2* w,
                            long long N, int nv, int nrhs, double sign, int split, cudaStream_t s);
// out = in * scale[rhs] written in the split form; the split form's FP32 rounding (h + l)
cudaError_t launch_scale_split(const double2* in, double2* out, const double* inv, long long N, int nrhs,
                               cudaStream_t s);
cudaError_t launch_split_to_f32(const double2* in, float2* out, long long n, cudaStream_t s);
cudaError_t launch_norm2_ds(const double2* w, long long N, int nrhs, double* part, double* out, int nblk,
                            cudaStream_t s);
// FGMRES Arnoldi bookkeeping on the device (one thread per rhs), see vec.cu
struct ArnoldiArgs {
  const double2* h;   // [rhs][j + 2]: Gram-Schmidt coefficients, then ||w||^2 before the pass
  const double* nrm;  // [rhs] ||w||^2 after the pass
  double2* H;         // [rhs][m][m + 1] Hessenberg columns (column-major)
  double2* cs;        // [rhs][m] Givens rotations
  double2* sn;
  double2* g;         // [rhs][m + 1] rotated residual vector
  const double* fn;   // [rhs] ||f||
  int* active;        // [rhs] 1 while the rhs iterates
  double* scal;       // [rhs] out: 1 / h_{j+1,j} (0 if inactive)
  double* stat;       // [rhs][5] out: active, steps, severe cancellation, non-finite, |g_{j+1}| / ||f||
  double tol;
  int nrhs, m;
};
cudaError_t launch_arnoldi(const ArnoldiArgs& a, int j, cudaStream_t s);
// out[rhs] = in[rhs] * scale[rhs] (real scale per rhs from a device array; 0 if scale is not finite)
cudaError_t launch_scale_rhs(const double2* in, double2* out, const double* inv, long long N, int nrhs,
                             cudaStream_t s);

}  // namespace th
