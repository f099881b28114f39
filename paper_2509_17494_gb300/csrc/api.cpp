// C ABI of the two-grid Helmholtz library: context, workspace, set-up upload,
// the two-grid cycle (Algorithm 1 with the CSDD smoother of Algorithm 2) and
// the outer right-preconditioned flexible GMRES.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "launch.cuh"
#include "unet_net.h"
#include "th_internal.h"

using th::cplx;

namespace {

// Bump allocator over the caller's workspace; with base == nullptr it only
// measures (th_workspace_size and th_setup carve in the same order).
struct Carve {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  bool ok = true;
  template <typename T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~(size_t)255;
    size_t bytes = count * sizeof(T);
    used = off + bytes;
    if (!base) return nullptr;
    if (used > cap) { ok = false; return nullptr; }
    return reinterpret_cast<T*>(base + off);
  }
};

inline bool has_prec(unsigned mask, int p) { return (mask >> p) & 1u; }

}  // namespace

struct th_ctx {
  th_mesh mesh{};
  th_params prm{};
  th::Geometry g;
  th::Ref1D ref;
  unsigned avail = 0;  // bitmask of prepared precisions
  int active = 0;
  bool mixed = false;  // any FP32-cycle precision prepared
  long long launches = 0;
  int cluster = 8, rpc = 0;
  int nblk = 1;
  int rmax = 0;
  int wchunks[4] = {0, 0, 0, 0};
  int ddG = 4;  // column groups per subdomain in K3
  int tc64 = 0, tc32 = 0;  // fine-apply tile variant per precision (0 large, 1 small), autotuned at 1 rhs
  int tcds = 0;            // the same for the double-single apply
  int tc64m = 0, tc32m = 0, tcdsm = 0;  // ... and at nrhs_max (>= 8) right-hand sides
  int dds64 = 0, dds32 = 0;  // DD kernel per precision: 0 k_dd_apply, 1 k_dd_stream (autotuned)
  int dd_tc = 1;             // batched BF16 products on tensor cores (k_dd_umma) when available
  int cs_variant = 1;        // one-rhs coarse chunk sweep: 0 two-phase, 1 one barrier per step (autotuned)
  int fuse = 1;              // cycle with u = 0 on entry: combine, prolongation and widening fused (TH_K_CYCLE)
  int cs_multi = 1;          // 8 or more right-hand sides: 0 per-tile cluster sweep, 1 column groups (TH_K_COARSE_MULTI)
  int coarse_refine = 0;     // mixed 2-D coarse solve: refinement steps on its FP32 residual (TH_K_COARSE_REFINE)
  int krylov_ds = 1;         // mixed forms' FGMRES dots, norms and updates: 1 double-single arithmetic, 0 FP64 (TH_K_KRYLOV)
  int sep_sym = 1;           // one-rhs FP32 separator product from Sinv's upper triangle (TH_K_SEP_SYM)
  unsigned char* Wu = nullptr;  // BF16 inverse rows in the tcgen05 operand layout (NR <= 128)
  int sms = 152;
  int device = -1;          // CUDA device the context was set up on
  int* derr = nullptr;      // device flag: a bounded device wait gave up
  // device arrays
  double *kc64 = nullptr, *ec64 = nullptr;
  float *kc32 = nullptr, *ec32 = nullptr;
  th::ds *kcds = nullptr, *ecds = nullptr;  // k, eps per cell in double-single (mixed form, 2-D)
  int resid_ds = 1;  // mixed form's outer residual: 1 double-single apply to FP32, 0 FP64 apply + rounding
  int az_ds = 1;     // mixed form's FGMRES product A z: 1 double-single apply with FP64 output, 0 FP64 apply
  int* box = nullptr;
  int4* ctab = nullptr;
  void* W[4] = {nullptr, nullptr, nullptr, nullptr};
  float* wscale16 = nullptr;
  int *pj0 = nullptr, *ridx = nullptr;
  double *pw64 = nullptr, *rw64 = nullptr;
  float *pw32 = nullptr, *rw32 = nullptr;
  double2 *ccell64 = nullptr, *crho64 = nullptr;
  float2 *ccell32 = nullptr, *crho32 = nullptr;
  double2 *G64 = nullptr, *cl64 = nullptr, *cd64 = nullptr, *cu64 = nullptr;  // G64: unpartitioned (no-alloc path)
  float2 *cl32 = nullptr, *cd32 = nullptr, *cu32 = nullptr;
  // partitioned coarse factors (both precisions when prepared)
  int P = 1, mcp = 0, Lmax = 0;
  int *ca = nullptr, *cb = nullptr, *sep = nullptr, *chunk_of = nullptr;
  int nred = 0;  // (P - 1) mc separator unknowns
  double2 *Gp64 = nullptr, *LR64 = nullptr, *Si64 = nullptr, *rh64 = nullptr;
  float2 *Gp32 = nullptr, *LR32 = nullptr, *Si32 = nullptr, *rh32 = nullptr;
  // 3-D coarse blocks (z-slices), sweep scratch and the fine apply's per-cell outputs
  double2 *G3_64 = nullptr, *dn64 = nullptr, *up64 = nullptr, *tsw64 = nullptr, *ycell64 = nullptr;
  float2 *G3_32 = nullptr, *dn32 = nullptr, *up32 = nullptr, *tsw32 = nullptr, *ycell32 = nullptr;
  // G_j transposed with rows padded to mcr, for the many-right-hand-side sweep (nrhs_max >= 2)
  int rpcm = 0, mcr = 0;
  double2* Gt64 = nullptr;
  float2* Gt32 = nullptr;
  float2* LRt32 = nullptr;  // spikes transposed ([j][col][mcr]) for the grouped FP32 spike correction (nrhs_max >= 8)
  // tensor-core separator product and spike correction (mixed 2-D, nrhs_max >= 8, P > 1): BF16 reduced
  // inverse and spikes in 128-row tiles of 64-column operand chunks, their tile tables and the BF16
  // operand staging of the reduced right-hand sides and separator values (coarse_umma.cu)
  unsigned char *Sb16 = nullptr, *LRb16 = nullptr, *rst16 = nullptr, *xst16 = nullptr;
  th::CoarseTile *tiles_s = nullptr, *tiles_l = nullptr;
  int ntiles_s = 0, ntiles_l = 0, nkc_s = 0, nkc_m = 0;
  int nsplit_s = 1;          // K splits of the separator product (to fill the SMs), partials in spart_s
  float2* spart_s = nullptr;
  long long lrb_chunks = 0;  // A chunks of the spikes over all tiles
  // one right-hand side (mixed 2-D): the upper-triangle 64 x 64 blocks of the reduced inverse, their
  // tile pairs and the partial products (k_sep_sym)
  float2 *Ssym32 = nullptr, *spart32 = nullptr;
  int2* sym_ij = nullptr;
  int Tsym = 0, nsym = 0;
  th::CoarseUmmaArgs umma{};
  // cycle work vectors
  double2 *r64 = nullptr, *s64 = nullptr, *v64 = nullptr, *V64 = nullptr, *rc64 = nullptr, *uc64 = nullptr,
          *zc64 = nullptr, *t64 = nullptr;
  float2 *f32 = nullptr, *u32 = nullptr, *r32 = nullptr, *s32 = nullptr, *v32 = nullptr, *V32 = nullptr,
         *rc32 = nullptr, *uc32 = nullptr, *zc32 = nullptr, *wc32 = nullptr;
  // FGMRES
  double2 *Vk = nullptr, *Zk = nullptr, *w = nullptr, *h1 = nullptr, *h2 = nullptr, *ybuf = nullptr,
          *dpart = nullptr;
  double *npart = nullptr, *nrm = nullptr, *scal = nullptr;
  // device-side Arnoldi state (Hessenberg columns, rotations, g, ||f||, flags, status)
  double2 *Hd = nullptr, *csd = nullptr, *snd = nullptr, *gd = nullptr;
  double *fnd = nullptr, *statd = nullptr;
  int* actd = nullptr;
  double* pin = nullptr;  // pinned host ring for the lagged status reads (allocated by th_solve)
  double2 *fin = nullptr, *uin = nullptr;  // device staging for the host-buffer entry points
  // per-kernel event timing (th_profile)
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> prof_rec;  // (kind, first event index)
  size_t ev_used = 0;
  // captured launch sequences (th_cycle_graph, the FGMRES preconditioner)
  struct Graph {
    int kind, nrhs, active;
    const void* a;
    const void* b;
    long long epoch, launches;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  cudaStream_t gstream = nullptr;  // private capture stream (the legacy stream cannot be captured)
  bool use_graphs = true;
  long long epoch = 0;  // bumped whenever a setting that changes the launch sequence changes
  // Galerkin p-type coarsening (coarse_kind TH_CK_GALERKIN): stencil and block inverses
  bool gal = false;
  double2 *gst64 = nullptr, *gG64 = nullptr;
  float2 *gst32 = nullptr, *gG32 = nullptr;
  // coarse correction: 0 direct solve, 1 learned corrector, 2 none; fallback count for th_solve
  int coarse_mode = 0, plain_iters = 0;
  th::UNet* unet = nullptr;
  std::vector<double> k_host;  // k per fine cell (inputs of the learned corrector)
  void drop_graphs() {
    for (Graph& gr : graphs) cudaGraphExecDestroy(gr.exec);
    graphs.clear();
  }
  ~th_ctx() {
    if (pin) cudaFreeHost(pin);
    delete unet;
    drop_graphs();
    if (gstream) cudaStreamDestroy(gstream);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  }
};

namespace {

th_status cuda_status(cudaError_t e) { return e == cudaSuccess ? TH_OK : TH_ERR_CUDA; }
// RAII bracket of one kernel launch with two events (only while profiling).
struct Prof {
  th_ctx& x;
  cudaStream_t s;
  int idx = -1;
  Prof(th_ctx& x_, int kind, cudaStream_t s_) : x(x_), s(s_) {
    if (!x.prof_on) return;
    if (x.ev_used + 2 > 65536) return;
    while (x.ev_pool.size() < x.ev_used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      x.ev_pool.push_back(e);
    }
    idx = (int)x.ev_used;
    x.ev_used += 2;
    cudaEventRecord(x.ev_pool[idx], s);
    x.prof_rec.push_back({kind, idx});
  }
  ~Prof() {
    if (idx >= 0) cudaEventRecord(x.ev_pool[idx + 1], s);
  }
};

#define TH_CU(expr)                                   \
  do {                                                \
    cudaError_t _e = (expr);                          \
    if (_e != cudaSuccess) return TH_ERR_CUDA;        \
  } while (0)

// Carves every device array in a fixed order (sizes only when c.base == nullptr).
void carve_all(th_ctx& x, Carve& c) {
  const th::Geometry& g = x.g;
  const th_params& prm = x.prm;
  const bool d3 = g.dim == 3;
  const size_t n2 = (size_t)g.n * g.n * (d3 ? g.n : 1);  // cells
  const int nr = prm.nrhs_max;
  x.derr = c.take<int>(64);
  x.kc64 = c.take<double>(n2);
  x.ec64 = c.take<double>(n2);
  x.box = c.take<int>((size_t)g.nsub * th::kBox);
  x.ctab = c.take<int4>((size_t)g.m);
  x.pj0 = c.take<int>(g.m);
  x.pw64 = c.take<double>((size_t)g.m * (g.q + 1));
  x.ridx = c.take<int>((size_t)g.mc * x.rmax);
  x.rw64 = c.take<double>((size_t)g.mc * x.rmax);
  const size_t ncell_c = d3 ? (size_t)g.nc * g.nc * g.nc * 4 : (size_t)g.nc * g.nc * 3;
  const size_t nrho_c = d3 ? (size_t)6 * g.nc * g.nc : (size_t)4 * g.nc;
  const size_t mb = (size_t)g.mc * g.mc;  // 3-D: nodes per z-slice
  x.ccell64 = c.take<double2>(ncell_c);
  x.crho64 = c.take<double2>(nrho_c);
  const size_t mm = (size_t)g.mc * g.mc;
  x.cl64 = c.take<double2>(mm);
  x.cd64 = c.take<double2>(mm);
  x.cu64 = c.take<double2>(mm);
  const int CPC[4] = {1, 2, 4, 4};
  for (int k = 0; k < 4; ++k) {
    x.wchunks[k] = (g.NC + CPC[k] - 1) / CPC[k];
    x.W[k] = has_prec(x.avail, k) ? (void*)c.take<uint4>((size_t)g.nsub * x.wchunks[k] * g.NR) : nullptr;
  }
  x.wscale16 = has_prec(x.avail, TH_PREC_FP16) ? c.take<float>(g.nsub) : nullptr;
  x.Wu = (has_prec(x.avail, TH_PREC_BF16) && g.NR <= 128 && prm.nrhs_max >= 8)
             ? c.take<unsigned char>((size_t)g.nsub * th::dd_umma_bytes_per_sub(g.NR, g.NC))
             : nullptr;
  const bool fp64 = has_prec(x.avail, TH_PREC_FP64);
  const bool qs = !x.gal;  // QSFEM coarse factors
  x.G64 = (fp64 && !d3 && qs) ? c.take<double2>(mm * g.mc) : nullptr;
  if (x.gal) {
    const size_t S = 2 * g.q + 1;
    const size_t gtot = (size_t)th::gal_goff(g.n, g.q, g.mc);
    x.gst64 = c.take<double2>((size_t)g.Nc * S * S);
    x.gG64 = fp64 ? c.take<double2>(gtot) : nullptr;
    if (x.mixed) {
      x.gst32 = c.take<float2>((size_t)g.Nc * S * S);
      x.gG32 = c.take<float2>(gtot);
    }
  }
  if (d3) {
    x.dn64 = c.take<double2>((size_t)g.mc * mb * 9);
    x.up64 = c.take<double2>((size_t)g.mc * mb * 9);
    x.G3_64 = fp64 ? c.take<double2>((size_t)g.mc * mb * mb) : nullptr;
    x.tsw64 = c.take<double2>((size_t)nr * mb);
    x.ycell64 = c.take<double2>((size_t)nr * n2 * 32);
    if (x.mixed) {
      x.dn32 = c.take<float2>((size_t)g.mc * mb * 9);
      x.up32 = c.take<float2>((size_t)g.mc * mb * 9);
      x.G3_32 = c.take<float2>((size_t)g.mc * mb * mb);
      x.tsw32 = c.take<float2>((size_t)nr * mb);
      x.ycell32 = c.take<float2>((size_t)nr * n2 * 32);
    }
  }
  const size_t blk = (size_t)g.mc * x.mcp;  // one padded dense block
  const int K = std::max(x.P - 1, 1);
  x.ca = c.take<int>(x.P);
  x.cb = c.take<int>(x.P);
  x.sep = c.take<int>(K);
  x.chunk_of = c.take<int>(g.mc);
  const size_t nred = std::max(x.nred, 1);
  if (fp64 && !d3 && qs) {
    x.Gp64 = c.take<double2>(blk * g.mc);
    x.LR64 = c.take<double2>(2 * blk * g.mc);
    x.Si64 = c.take<double2>(nred * (nred + (nred & 1)));
    x.rh64 = c.take<double2>(nred * nr);
    if (nr >= 2) x.Gt64 = c.take<double2>(mm * x.mcr);
  }
  // FP64 work vectors are always present (residuals, FGMRES, FP64 applies)
  x.r64 = c.take<double2>((size_t)nr * g.N);
  x.s64 = c.take<double2>((size_t)nr * g.N);
  x.v64 = c.take<double2>((size_t)nr * g.N);
  x.t64 = c.take<double2>((size_t)nr * g.N);
  x.V64 = fp64 ? c.take<double2>((size_t)nr * g.nsub * g.NR) : nullptr;
  x.rc64 = c.take<double2>((size_t)nr * g.Nc);
  x.uc64 = c.take<double2>((size_t)nr * g.Nc);

  if (x.mixed) {
    x.kc32 = c.take<float>(n2);
    x.ec32 = c.take<float>(n2);
    x.kcds = c.take<th::ds>(n2);
    x.ecds = c.take<th::ds>(n2);
    x.pw32 = c.take<float>((size_t)g.m * (g.q + 1));
    x.rw32 = c.take<float>((size_t)g.mc * x.rmax);
    x.ccell32 = c.take<float2>(ncell_c);
    x.crho32 = c.take<float2>(nrho_c);
    x.cl32 = c.take<float2>(mm);
    x.cd32 = c.take<float2>(mm);
    x.cu32 = c.take<float2>(mm);
    if (!d3 && qs) {
      x.Gp32 = c.take<float2>(blk * g.mc);
      x.LR32 = c.take<float2>(2 * blk * g.mc);
      x.Si32 = c.take<float2>(nred * (nred + (nred & 1)));
      x.rh32 = c.take<float2>(nred * nr);
      if (nr >= 2) x.Gt32 = c.take<float2>(mm * x.mcr);
      if (nr >= 8) x.LRt32 = c.take<float2>((size_t)g.mc * 2 * x.mcp * x.mcr);
      if (x.P > 1) {
        x.Tsym = (x.nred + 63) / 64;
        x.nsym = x.Tsym * (x.Tsym + 1) / 2;
        x.Ssym32 = c.take<float2>((size_t)x.nsym * 64 * 64);
        x.sym_ij = c.take<int2>((size_t)x.nsym);
        x.spart32 = c.take<float2>((size_t)x.Tsym * x.Tsym * 64);
      }
      if (nr >= 8 && x.P > 1) {
        // chunk lengths of coarse_partition (P - 1 separator rows between P chunks)
        const int rows = g.mc - (x.P - 1), base = rows / x.P, rem = rows % x.P;
        x.nkc_s = (x.nred + 31) / 32;
        x.nkc_m = (g.mc + 31) / 32;
        x.ntiles_s = (x.nred + 127) / 128;
        x.ntiles_l = 0;
        x.lrb_chunks = 0;
        for (int ch = 0; ch < x.P; ++ch) {
          const long long L = base + (ch < rem ? 1 : 0);
          const int t = (int)((L * g.mc + 127) / 128);
          const int sides = (ch > 0 ? 1 : 0) + (ch < x.P - 1 ? 1 : 0);
          x.ntiles_l += t;
          x.lrb_chunks += (long long)t * sides * x.nkc_m;
        }
        const size_t groups = (size_t)(nr + 63) / 64;
        x.Sb16 = c.take<unsigned char>((size_t)x.ntiles_s * x.nkc_s * 32768);
        x.LRb16 = c.take<unsigned char>((size_t)x.lrb_chunks * 32768);
        x.rst16 = c.take<unsigned char>(groups * x.nkc_s * 16384);
        x.xst16 = c.take<unsigned char>(groups * (x.P - 1) * x.nkc_m * 16384);
        // split the separator product over K so that its tiles fill the 152 SMs (the tiles of
        // the 401-row grid: 60), at least 8 chunks a split
        x.nsplit_s = std::max(1, std::min(std::min(8, 152 / std::max(1, x.ntiles_s)), x.nkc_s / 8));
        x.tiles_s = c.take<th::CoarseTile>((size_t)x.ntiles_s * x.nsplit_s);
        x.spart_s = x.nsplit_s > 1 ? c.take<float2>((size_t)x.nsplit_s * groups * 64 * x.nred) : nullptr;
        x.tiles_l = c.take<th::CoarseTile>(x.ntiles_l);
      }
    }
    x.f32 = c.take<float2>((size_t)nr * g.N);
    x.u32 = c.take<float2>((size_t)nr * g.N);
    x.r32 = c.take<float2>((size_t)nr * g.N);
    x.s32 = c.take<float2>((size_t)nr * g.N);
    x.v32 = c.take<float2>((size_t)nr * g.N);
    x.V32 = c.take<float2>((size_t)nr * g.nsub * g.NR);
    x.rc32 = c.take<float2>((size_t)nr * g.Nc);
    x.uc32 = c.take<float2>((size_t)nr * g.Nc);
    if (!d3 && qs) {  // coarse residual and correction of the refinement steps
      x.zc32 = c.take<float2>((size_t)nr * g.Nc);
      x.wc32 = c.take<float2>((size_t)nr * g.Nc);
    }
  }
  const int m = prm.restart;
  x.Vk = c.take<double2>((size_t)(m + 1) * nr * g.N);
  x.Zk = c.take<double2>((size_t)m * nr * g.N);
  x.w = c.take<double2>((size_t)nr * g.N);
  x.h1 = c.take<double2>((size_t)nr * (m + 1));
  x.h2 = c.take<double2>((size_t)nr * (m + 1));
  x.ybuf = c.take<double2>((size_t)nr * (m + 1));
  x.nblk = th::mdot_blocks(g.N);
  x.dpart = c.take<double2>((size_t)nr * (m + 1) * x.nblk);
  x.npart = c.take<double>((size_t)nr * x.nblk);
  x.nrm = c.take<double>((size_t)nr);
  x.scal = c.take<double>((size_t)nr);
  x.Hd = c.take<double2>((size_t)nr * (m + 1) * m);
  x.csd = c.take<double2>((size_t)nr * m);
  x.snd = c.take<double2>((size_t)nr * m);
  x.gd = c.take<double2>((size_t)nr * (m + 1));
  x.fnd = c.take<double>((size_t)nr);
  x.statd = c.take<double>((size_t)nr * 5);
  x.actd = c.take<int>((size_t)nr);
  x.fin = c.take<double2>((size_t)nr * g.N);
  x.uin = c.take<double2>((size_t)nr * g.N);
}

th_status prepare(const th_mesh* mesh, const th_params* prm, th_ctx& x) {
  if (!mesh || !prm) return TH_ERR_ARG;
  x.mesh = *mesh;
  x.prm = *prm;
  th_status st = th::make_geometry(*mesh, *prm, x.g);
  if (st != TH_OK) return st;
  if (prm->coarse_kind != TH_CK_QSFEM && prm->coarse_kind != TH_CK_GALERKIN) return TH_ERR_ARG;
  if (!std::isfinite(prm->alpha_c) || prm->alpha_c < 0.0) return TH_ERR_ARG;
  x.gal = prm->coarse_kind == TH_CK_GALERKIN;
  if (x.gal && x.g.dim != 2) return TH_ERR_UNSUPPORTED;
  if (x.gal && (x.g.dirichlet[0] | x.g.dirichlet[1] | x.g.dirichlet[2] | x.g.dirichlet[3]))
    return TH_ERR_UNSUPPORTED;  // Galerkin coarsening with Dirichlet sides is not built
  // block 0 of the Galerkin sweep holds its right-hand side in shared memory
  if (x.gal && (size_t)(x.g.q + 1) * x.g.mc * 16 > 227 * 1024) return TH_ERR_UNSUPPORTED;
  if (x.g.dim == 2 && x.g.mc > 1024) return TH_ERR_UNSUPPORTED;  // coarse kernels hold two coarse rows per thread
  if (x.g.dim == 3 && (long long)x.g.mc * x.g.mc > 4096) return TH_ERR_UNSUPPORTED;  // z-slice blocks of mc^2 <= 4096
  x.avail = (prm->prec_mask & 0xFu) | (1u << prm->prec);
  x.active = prm->prec;
  x.mixed = (x.avail & ~1u) != 0;
  // restriction table width
  th::Ref1D ref = th::reference_1d(mesh->p);
  th::TransferTables tt;
  th::transfer_tables(x.g, ref, tt);
  x.rmax = tt.rmax;
  x.ref = ref;
  x.cluster = 8;
  x.rpc = (x.g.mc + x.cluster - 1) / x.cluster;
  if (prm->coarse_chunks < 0 || (prm->coarse_chunks > 0 && 2 * prm->coarse_chunks - 1 > x.g.mc)) return TH_ERR_ARG;
  x.P = x.g.dim == 2 ? (prm->coarse_chunks > 0 ? prm->coarse_chunks : th::coarse_chunks(x.g.mc)) : 1;
  x.mcp = x.g.mc + (x.g.mc & 1);
  x.rpcm = x.rpc + (x.rpc & 1);
  x.mcr = x.cluster * x.rpcm;
  {
    const int rows = x.g.mc - (x.P - 1);
    x.Lmax = rows / x.P + ((rows % x.P) ? 1 : 0);
    x.nred = (x.P - 1) * x.g.mc;
  }
  return TH_OK;
}

uint16_t f2bf(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);  // inf / nan
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// a complex value as four BF16 parts (re hi, im hi, re lo, im lo), `part` entries apart:
// v = hi + lo with hi = bf16(v), lo = bf16(v - hi), both rounded to nearest
void put_split(uint16_t* dst, int off, int part, cplx v) {
  const double re = v.real(), im = v.imag();
  const uint16_t hr = f2bf((float)re), hi = f2bf((float)im);
  auto up = [](uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
  };
  dst[off] = hr;
  dst[part + off] = hi;
  dst[2 * part + off] = f2bf((float)(re - up(hr)));
  dst[3 * part + off] = f2bf((float)(im - up(hi)));
}

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

template <typename T>
T cvt(double v) {
  if constexpr (std::is_same<T, th::ds>::value) return th::ds_from_host(v);
  else return (T)v;
}

// the autotuned tile variant of the fine apply for precision T and nrhs right-hand sides
template <typename T>
int fine_tile(const th_ctx& x, int nrhs) {
  const bool many = nrhs >= 8;
  if constexpr (std::is_same<T, float>::value) return many ? x.tc32m : x.tc32;
  else if constexpr (std::is_same<T, th::ds>::value) return many ? x.tcdsm : x.tcds;
  else return many ? x.tc64m : x.tc64;
}

template <typename T>
th::FineArgs<T> fine_args(const th_ctx& x, int op, int nrhs) {
  th::FineArgs<T> a{};
  const th::Geometry& g = x.g;
  a.N = g.N;
  a.n = g.n;
  a.m = g.m;
  a.p = g.p;
  a.robin = g.robin[0] | (g.robin[1] << 1) | (g.robin[2] << 2) | (g.robin[3] << 3);
  a.dirichlet = g.dirichlet[0] | (g.dirichlet[1] << 1) | (g.dirichlet[2] << 2) | (g.dirichlet[3] << 3);
  a.h = cvt<T>(g.h);
  a.h2 = cvt<T>(g.h * g.h);
  a.alpha = cvt<T>(op == TH_OP_AS ? x.prm.alpha_s : 0.0);
  a.tc = fine_tile<T>(x, nrhs);
  const int np = g.p + 1;
  for (int i = 0; i < np * np; ++i) {
    a.M[i] = cvt<T>(x.ref.M[i]);
    a.K[i] = cvt<T>(x.ref.K[i]);
  }
  const int H = g.p / 2, P = g.p;
  const double* M = x.ref.M.data();
  const double* K = x.ref.K.data();
  for (int r = 0; r <= H; ++r)
    for (int c = 0; c <= H; ++c) {
      const bool mid = (c == H);
      a.ME[r * (H + 1) + c] = cvt<T>(mid ? M[r * np + c] : 0.5 * (M[r * np + c] + M[r * np + P - c]));
      a.KE[r * (H + 1) + c] = cvt<T>(mid ? K[r * np + c] : 0.5 * (K[r * np + c] + K[r * np + P - c]));
    }
  for (int r = 0; r < H; ++r)
    for (int c = 0; c < H; ++c) {
      a.MO[r * H + c] = cvt<T>(0.5 * (M[r * np + c] - M[r * np + P - c]));
      a.KO[r * H + c] = cvt<T>(0.5 * (K[r * np + c] - K[r * np + P - c]));
    }
  if constexpr (std::is_same<T, double>::value) {
    a.kc = x.kc64;
    a.ec = x.ec64;
  } else if constexpr (std::is_same<T, th::ds>::value) {
    a.kc = x.kcds;
    a.ec = x.ecds;
  } else {
    a.kc = x.kc32;
    a.ec = x.ec32;
  }
  return a;
}

// y = OP u or y = f - OP u, in precision T, on nrhs right-hand sides
template <typename T>
th_status fine_apply3(th_ctx& x, int op, const typename th::Cx<T>::t* u, const typename th::Cx<T>::t* f,
                      typename th::Cx<T>::t* y, int nrhs, cudaStream_t s) {
  const th::Geometry& g = x.g;
  th::Fine3Args<T> a{};
  a.u = u;
  a.f = f;
  a.y = y;
  a.residual = f ? 1 : 0;
  a.N = g.N;
  a.ncell = (long long)g.n * g.n * g.n;
  a.n = g.n;
  a.m = g.m;
  a.robin = 0;
  for (int s6 = 0; s6 < 6; ++s6) a.robin |= g.robin[s6] << s6;
  a.h = cvt<T>(g.h);
  a.alpha = cvt<T>(op == TH_OP_AS ? x.prm.alpha_s : 0.0);
  for (int i = 0; i < 9; ++i) {
    a.M[i] = cvt<T>(x.ref.M[i]);
    a.K[i] = cvt<T>(x.ref.K[i]);
  }
  if constexpr (std::is_same<T, double>::value) {
    a.kc = x.kc64;
    a.ec = x.ec64;
    a.ycell = x.ycell64;
  } else if constexpr (std::is_same<T, th::ds>::value) {
    a.kc = x.kcds;
    a.ec = x.ecds;
    a.ycell = reinterpret_cast<th::cds*>(x.ycell64);  // 16-byte entries, as FP64
  } else {
    a.kc = x.kc32;
    a.ec = x.ec32;
    a.ycell = x.ycell32;
  }
  if (!a.ycell) return TH_ERR_UNSUPPORTED;
  x.launches += 2;
  Prof prof(x, TH_K_FINE, s);
  return cuda_status(th::launch_fine3<T>(a, nrhs, s));
}

template <typename T>
th_status fine_apply(th_ctx& x, int op, const typename th::Cx<T>::t* u, const typename th::Cx<T>::t* f,
                     typename th::Cx<T>::t* y, int nrhs, cudaStream_t s) {
  if (x.g.dim == 3) return fine_apply3<T>(x, op, u, f, y, nrhs, s);
  th::FineArgs<T> a = fine_args<T>(x, op, nrhs);
  a.u = u;
  a.f = f;
  a.y = y;
  a.residual = f ? 1 : 0;
  x.launches += 1;
  Prof prof(x, TH_K_FINE, s);
  return cuda_status(th::launch_fine_apply<T>(a, nrhs, s));
}

// The mixed form's outer residual r = f - A u from FP64 u, f, delivered in FP32
// (the FP32 cycle's input): a double-single apply that writes FP32 (one launch),
// or the FP64 apply followed by rounding (th_set_kernel_variant TH_K_RESID).
th_status outer_residual(th_ctx& x, const double2* u, const double2* f, float2* r32, int nrhs, cudaStream_t s) {
  if (x.g.dim == 3 && x.resid_ds && x.kcds)  // double-single 3-D apply, FP32 output (see NodeIO<ds>)
    return fine_apply3<th::ds>(x, TH_OP_A, reinterpret_cast<const th::cds*>(u), reinterpret_cast<const th::cds*>(f),
                               reinterpret_cast<th::cds*>(r32), nrhs, s);
  if (x.g.dim == 2 && x.resid_ds && x.kcds) {
    th::FineArgs<th::ds> a = fine_args<th::ds>(x, TH_OP_A, nrhs);
    a.u = reinterpret_cast<const th::cds*>(u);
    a.f = reinterpret_cast<const th::cds*>(f);
    a.y = reinterpret_cast<th::cds*>(r32);  // FP32 output (see NodeIO<ds>)
    a.residual = 1;
    x.launches += 1;
    Prof prof(x, TH_K_FINE, s);
    return cuda_status(th::launch_fine_apply<th::ds>(a, nrhs, s));
  }
  th_status st = fine_apply<double>(x, TH_OP_A, u, f, x.r64, nrhs, s);
  if (st != TH_OK) return st;
  x.launches += 1;
  Prof prof(x, TH_K_VECTOR, s);
  return cuda_status(th::launch_d2f((const double*)x.r64, (float*)r32, 2 * x.g.N * (long long)nrhs, s));
}

// The FGMRES product w = A z.  In the mixed forms (2-D) it runs in double-single
// arithmetic (48-bit significands, 64-bit exponent range of FP32 pairs) with
// FP64 output, TH_K_AZ 1: GB300's FP64 rate is 1/64 of its FP32 rate; the
// Arnoldi relation then holds to ~1e-14 relative, far below the 1e-8
// tolerance, and the final residual is recomputed in FP64.
th_status az_apply(th_ctx& x, const double2* z, double2* w, int nrhs, cudaStream_t s) {
  if (x.active != TH_PREC_FP64 && x.az_ds && x.kcds && x.g.dim == 2) {
    th::FineArgs<th::ds> a = fine_args<th::ds>(x, TH_OP_A, nrhs);
    a.u = reinterpret_cast<const th::cds*>(z);
    a.f = nullptr;
    a.y = reinterpret_cast<th::cds*>(w);
    a.residual = 0;
    a.out64 = 1;
    x.launches += 1;
    Prof prof(x, TH_K_FINE, s);
    return cuda_status(th::launch_fine_apply<th::ds>(a, nrhs, s));
  }
  return fine_apply<double>(x, TH_OP_A, z, nullptr, w, nrhs, s);
}

// r = f - A u into an FP64 vector: in double-single arithmetic where the mixed
// form's double-single apply exists (exact = false), else FP64.  th_solve takes
// its restart residuals this way and confirms convergence with the FP64 apply.
th_status fgmres_residual(th_ctx& x, const double2* u, const double2* f, double2* r, int nrhs, cudaStream_t s,
                          bool exact) {
  if (!exact && x.active != TH_PREC_FP64 && x.az_ds && x.kcds && x.g.dim == 2) {
    th::FineArgs<th::ds> a = fine_args<th::ds>(x, TH_OP_A, nrhs);
    a.u = reinterpret_cast<const th::cds*>(u);
    a.f = reinterpret_cast<const th::cds*>(f);
    a.y = reinterpret_cast<th::cds*>(r);
    a.residual = 1;
    a.out64 = 1;
    x.launches += 1;
    Prof prof(x, TH_K_FINE, s);
    return cuda_status(th::launch_fine_apply<th::ds>(a, nrhs, s));
  }
  return fine_apply<double>(x, TH_OP_A, u, f, r, nrhs, s);
}

template <typename T> struct PrecBufs;
template <> struct PrecBufs<double> {
  static double2* r(th_ctx& x) { return x.r64; }
  static double2* s(th_ctx& x) { return x.s64; }
  static double2* v(th_ctx& x) { return x.v64; }
  static double2* V(th_ctx& x) { return x.V64; }
  static double2* rc(th_ctx& x) { return x.rc64; }
  static double2* uc(th_ctx& x) { return x.uc64; }
  static const double2* Gp(th_ctx& x) { return x.Gp64; }
  static const double2* Gt(th_ctx& x) { return x.Gt64; }
  static const double2* LR(th_ctx& x) { return x.LR64; }
  static const double2* Si(th_ctx& x) { return x.Si64; }
  static double2* rh(th_ctx& x) { return x.rh64; }
  static const double* pw(th_ctx& x) { return x.pw64; }
  static const double* rw(th_ctx& x) { return x.rw64; }
  static const double2* cl(th_ctx& x) { return x.cl64; }
  static const double2* cd(th_ctx& x) { return x.cd64; }
  static const double2* cu(th_ctx& x) { return x.cu64; }
  static const double2* cell(th_ctx& x) { return x.ccell64; }
  static const double2* rho(th_ctx& x) { return x.crho64; }
  static const double2* G3(th_ctx& x) { return x.G3_64; }
  static const double2* dn(th_ctx& x) { return x.dn64; }
  static const double2* up(th_ctx& x) { return x.up64; }
  static double2* tsw(th_ctx& x) { return x.tsw64; }
  static double2* ycell(th_ctx& x) { return x.ycell64; }
};
template <> struct PrecBufs<float> {
  static float2* r(th_ctx& x) { return x.r32; }
  static float2* s(th_ctx& x) { return x.s32; }
  static float2* v(th_ctx& x) { return x.v32; }
  static float2* V(th_ctx& x) { return x.V32; }
  static float2* rc(th_ctx& x) { return x.rc32; }
  static float2* uc(th_ctx& x) { return x.uc32; }
  static const float2* Gp(th_ctx& x) { return x.Gp32; }
  static const float2* Gt(th_ctx& x) { return x.Gt32; }
  static const float2* LR(th_ctx& x) { return x.LR32; }
  static const float2* Si(th_ctx& x) { return x.Si32; }
  static float2* rh(th_ctx& x) { return x.rh32; }
  static const float* pw(th_ctx& x) { return x.pw32; }
  static const float* rw(th_ctx& x) { return x.rw32; }
  static const float2* cl(th_ctx& x) { return x.cl32; }
  static const float2* cd(th_ctx& x) { return x.cd32; }
  static const float2* cu(th_ctx& x) { return x.cu32; }
  static const float2* cell(th_ctx& x) { return x.ccell32; }
  static const float2* rho(th_ctx& x) { return x.crho32; }
  static const float2* G3(th_ctx& x) { return x.G3_32; }
  static const float2* dn(th_ctx& x) { return x.dn32; }
  static const float2* up(th_ctx& x) { return x.up32; }
  static float2* tsw(th_ctx& x) { return x.tsw32; }
  static float2* ycell(th_ctx& x) { return x.ycell32; }
};

template <typename T>
th_status dd_apply(th_ctx& x, int wkind, const typename th::Cx<T>::t* r, int nrhs, cudaStream_t s) {
  using B = PrecBufs<T>;
  const th::Geometry& g = x.g;
  th::DDArgs<T> a{};
  a.r = r;
  a.V = B::V(x);
  a.W = x.W[wkind];
  a.box = x.box;
  a.wscale = (wkind == TH_PREC_FP16) ? x.wscale16 : nullptr;
  a.N = g.N;
  a.nsub = g.nsub;
  a.m = g.m;
  a.Lw = g.Lw;
  a.NC = g.NC;
  a.NCH = x.wchunks[wkind];
  a.NR = g.NR;
  a.G = std::max(1, std::min(x.ddG, 512 / std::max(1, g.NR)));  // boxes above 512 nodes: one group, 1024 threads
  a.nrhs = nrhs;
  x.launches += 1;
  Prof prof(x, TH_K_DD, s);
  if constexpr (std::is_same<T, float>::value) {
    if (wkind == TH_PREC_BF16 && x.Wu && x.dd_tc && nrhs >= 8) {
      th::DDUmmaArgs u{};
      u.r = r;
      u.V = a.V;
      u.W = x.Wu;
      u.box = x.box;
      u.err = x.derr;
      u.N = g.N;
      u.nsub = g.nsub;
      u.m = g.m;
      u.Lw = g.Lw;
      u.NC = g.NC;
      u.NR = g.NR;
      u.nrhs = nrhs;
      u.M8 = (g.NR + 7) / 8;
      u.K8 = 2 * ((g.NC + 15) / 16);
      u.dim3 = g.dim == 3 ? 1 : 0;
      return cuda_status(th::launch_dd_umma(u, x.sms, s));
    }
  }
  const int stream = std::is_same<T, double>::value ? x.dds64 : x.dds32;
  a.stream_v2 = stream == 2 ? 1 : 0;
  a.stream_small = (stream == 3 || stream == 5) ? 1 : 0;
  a.stream_pk = stream >= 4 ? 1 : 0;
  if (stream) return cuda_status(th::launch_dd_stream<T>(a, wkind, x.derr, x.sms, s));
  return cuda_status(th::launch_dd_apply<T>(a, wkind, 0, s));
}

template <typename T>
th_status dd_combine(th_ctx& x, typename th::Cx<T>::t* u, int accumulate, int nrhs, cudaStream_t s) {
  const th::Geometry& g = x.g;
  th::CombineArgs<T> a{};
  a.V = PrecBufs<T>::V(x);
  a.u = u;
  a.ctab = x.ctab;
  a.N = g.N;
  a.m = g.m;
  a.nb = g.nb;
  a.Lu = g.Lu;
  a.NR = g.NR;
  a.nsub = g.nsub;
  a.accumulate = accumulate;
  x.launches += 1;
  Prof prof(x, TH_K_COMBINE, s);
  if (g.dim == 3) return cuda_status(th::launch_dd_combine3<T>(a, nrhs, s));
  return cuda_status(th::launch_dd_combine<T>(a, nrhs, s));
}

// CSDDSmoother(u, f) of Algorithm 2 in precision T.  u_zero: u is known to be
// zero on entry (then r = f and u is overwritten).
template <typename T>
th_status smooth(th_ctx& x, int wkind, const typename th::Cx<T>::t* f, typename th::Cx<T>::t* u, bool u_zero,
                 int nrhs, cudaStream_t s) {
  using B = PrecBufs<T>;
  using C = typename th::Cx<T>::t;
  th_status st;
  const C* r = f;
  if (!u_zero) {
    if ((st = fine_apply<T>(x, TH_OP_A, u, f, B::r(x), nrhs, s)) != TH_OK) return st;
    r = B::r(x);
  }
  if ((st = dd_apply<T>(x, wkind, r, nrhs, s)) != TH_OK) return st;
  if (x.prm.n_dd == 1) return dd_combine<T>(x, u, u_zero ? 0 : 1, nrhs, s);
  // n_dd >= 2: v = DDStep(0, r); then v <- DDStep(v, r) = v + avg(W R (r - A_s v))
  C* v = B::v(x);
  if ((st = dd_combine<T>(x, v, 0, nrhs, s)) != TH_OK) return st;
  for (int it = 1; it < x.prm.n_dd; ++it) {
    if ((st = fine_apply<T>(x, TH_OP_AS, v, r, B::s(x), nrhs, s)) != TH_OK) return st;
    if ((st = dd_apply<T>(x, wkind, B::s(x), nrhs, s)) != TH_OK) return st;
    if ((st = dd_combine<T>(x, v, 1, nrhs, s)) != TH_OK) return st;
  }
  const long long n = x.g.N * (long long)nrhs;
  x.launches += 1;
  Prof prof(x, TH_K_VECTOR, s);
  if (u_zero) return cuda_status(cudaMemcpyAsync(u, v, sizeof(C) * n, cudaMemcpyDeviceToDevice, s));
  return cuda_status(th::launch_zaxpy<T>(v, u, (T)1, n, s));
}

template <typename T>
th_status restrict_(th_ctx& x, const typename th::Cx<T>::t* r, typename th::Cx<T>::t* rc, int nrhs, cudaStream_t s) {
  using B = PrecBufs<T>;
  th::TransferArgs<T> a{};
  a.in = r;
  a.out = rc;
  a.ridx = x.ridx;
  a.rw = B::rw(x);
  a.rmax = x.rmax;
  a.dirichlet = x.g.dirichlet[0] | (x.g.dirichlet[1] << 1) | (x.g.dirichlet[2] << 2) | (x.g.dirichlet[3] << 3);
  a.N = x.g.N;
  a.Nc = x.g.Nc;
  a.m = x.g.m;
  a.mc = x.g.mc;
  a.q = x.g.q;
  x.launches += 1;
  Prof prof(x, TH_K_RESTRICT, s);
  if (x.g.dim == 3) return cuda_status(th::launch_restrict3<T>(a, nrhs, s));
  return cuda_status(th::launch_restrict<T>(a, nrhs, s));
}

template <typename T>
th_status prolong_(th_ctx& x, const typename th::Cx<T>::t* uc, typename th::Cx<T>::t* u, T omega, int nrhs,
                   cudaStream_t s) {
  using B = PrecBufs<T>;
  th::TransferArgs<T> a{};
  a.in = uc;
  a.out = u;
  a.pj0 = x.pj0;
  a.pw = B::pw(x);
  a.N = x.g.N;
  a.Nc = x.g.Nc;
  a.m = x.g.m;
  a.mc = x.g.mc;
  a.q = x.g.q;
  a.omega = omega;
  a.dirichlet = x.g.dirichlet[0] | (x.g.dirichlet[1] << 1) | (x.g.dirichlet[2] << 2) | (x.g.dirichlet[3] << 3);
  x.launches += 1;
  Prof prof(x, TH_K_PROLONG, s);
  if (x.g.dim == 3) return cuda_status(th::launch_prolong3<T>(a, nrhs, s));
  return cuda_status(th::launch_prolong<T>(a, nrhs, s));
}

template <typename T>
th_status coarse_solve3_(th_ctx& x, const typename th::Cx<T>::t* rc, typename th::Cx<T>::t* uc, int nrhs,
                         cudaStream_t s) {
  using B = PrecBufs<T>;
  th::Sweep3Args<T> a{};
  a.b = rc;
  a.x = uc;
  a.t = B::tsw(x);
  a.G = B::G3(x);
  a.dn = B::dn(x);
  a.up = B::up(x);
  a.Nc = x.g.Nc;
  a.mc = x.g.mc;
  a.mb = x.g.mc * x.g.mc;
  a.nrhs = nrhs;
  if (!a.G || !a.t) return TH_ERR_UNSUPPORTED;
  x.launches += 4 * x.g.mc - 2;
  Prof prof(x, TH_K_COARSE_SOLVE, s);
  return cuda_status(th::launch_sweep3<T>(a, s));
}

template <typename T>
th::GalArgs<T> gal_args(th_ctx& x, const typename th::Cx<T>::t* in, typename th::Cx<T>::t* out, int nrhs) {
  th::GalArgs<T> a{};
  if constexpr (std::is_same<T, double>::value) {
    a.st = x.gst64;
    a.G = x.gG64;
  } else {
    a.st = x.gst32;
    a.G = x.gG32;
  }
  a.b = in;
  a.x = out;
  a.Nc = x.g.Nc;
  a.q = x.g.q;
  a.mc = x.g.mc;
  a.nblk = x.g.n;
  a.nrhs = nrhs;
  return a;
}

// Galerkin p-type coarsening: u_c = A_c^{-1} r_c by the block sweep
template <typename T>
th_status gal_solve_(th_ctx& x, const typename th::Cx<T>::t* rc, typename th::Cx<T>::t* uc, int nrhs,
                     cudaStream_t s) {
  const th::GalArgs<T> a = gal_args<T>(x, rc, uc, nrhs);
  if (!a.st || !a.G) return TH_ERR_UNSUPPORTED;
  x.launches += th::gal_solve_launches(a.nblk);
  Prof prof(x, TH_K_COARSE_SOLVE, s);
  return cuda_status(th::launch_gal_solve<T>(a, s));
}

template <typename T>
th_status coarse_solve_once_(th_ctx& x, const typename th::Cx<T>::t* rc, typename th::Cx<T>::t* uc, int nrhs,
                             cudaStream_t s) {
  if (x.g.dim == 3) return coarse_solve3_<T>(x, rc, uc, nrhs, s);
  if (x.gal) return gal_solve_<T>(x, rc, uc, nrhs, s);
  using B = PrecBufs<T>;
  th::CoarsePartArgs<T> a{};
  a.b = rc;
  a.x = uc;
  a.G = B::Gp(x);
  a.LR = B::LR(x);
  a.Sinv = B::Si(x);
  a.rhat = B::rh(x);
  a.nred = x.nred;
  a.ldS = x.nred + (x.nred & 1);
  a.cl = B::cl(x);
  a.cd = B::cd(x);
  a.cu = B::cu(x);
  a.ca = x.ca;
  a.cb = x.cb;
  a.sep = x.sep;
  a.chunk_of = x.chunk_of;
  a.Nc = x.g.Nc;
  a.mc = x.g.mc;
  a.mcp = x.mcp;
  a.P = x.P;
  a.rpc = x.rpc;
  a.Lmax = x.Lmax;
  a.Gt = B::Gt(x);
  if constexpr (std::is_same<T, float>::value) {
    a.LRt = x.LRt32;
    if (x.Sb16) {
      a.rst = x.rst16;
      a.nkc_s = x.nkc_s;
      a.umma = &x.umma;
    }
    if (x.sep_sym) {
      a.Ssym = x.Ssym32;
      a.sym_ij = x.sym_ij;
      a.spart = x.spart32;
      a.Tsym = x.Tsym;
      a.nsym = x.nsym;
    }
  }
  a.mcr = x.mcr;
  a.rpcm = x.rpcm;
  a.nrhs = nrhs;
  a.sweep_variant = x.cs_variant;
  a.multi_variant = x.cs_multi;
  a.nsm = x.sms;
  a.err = x.derr;
  if (!a.G || !a.LR) return TH_ERR_UNSUPPORTED;
  x.launches += (x.P > 1) ? ((nrhs == 1 && a.Ssym) ? 5 : 4) : 1;
  Prof prof(x, TH_K_COARSE_SOLVE, s);
  return cuda_status(th::launch_coarse_part<T>(a, nrhs, x.cluster, s));
}

// FP32 coarse residual z = r_c - A_q u_c (2-D QSFEM coarse level)
th_status coarse_residual32(th_ctx& x, const float2* rc, const float2* uc, float2* z, int nrhs, cudaStream_t s) {
  th::CoarseApplyArgs<float> a{};
  a.x = uc;
  a.y = z;
  a.f = rc;
  a.cell = x.ccell32;
  a.rho = x.crho32;
  a.Nc = x.g.Nc;
  a.nc = x.g.nc;
  a.mc = x.g.mc;
  a.dirichlet = x.g.dirichlet[0] | (x.g.dirichlet[1] << 1) | (x.g.dirichlet[2] << 2) | (x.g.dirichlet[3] << 3);
  x.launches += 1;
  Prof prof(x, TH_K_COARSE_APPLY, s);
  return cuda_status(th::launch_coarse_apply<float>(a, nrhs, s));
}

// The coarse solve of the cycle.  In FP32 the partitioned solve can lose
// several digits on large coarse grids (its chunk systems amplify rounding
// errors); there `coarse_refine` steps of iterative refinement follow it:
// z = r_c - A_q u_c in FP32, w = the same solve of z, u_c += w.
template <typename T>
th_status coarse_solve_(th_ctx& x, const typename th::Cx<T>::t* rc, typename th::Cx<T>::t* uc, int nrhs,
                        cudaStream_t s) {
  th_status st = coarse_solve_once_<T>(x, rc, uc, nrhs, s);
  if constexpr (std::is_same<T, float>::value) {
    if (st != TH_OK || x.coarse_refine <= 0 || x.g.dim != 2 || x.gal || !x.zc32 || !x.wc32) return st;
    for (int it = 0; it < x.coarse_refine; ++it) {
      if ((st = coarse_residual32(x, rc, uc, x.zc32, nrhs, s)) != TH_OK) return st;
      if ((st = coarse_solve_once_<T>(x, x.zc32, x.wc32, nrhs, s)) != TH_OK) return st;
      x.launches += 1;
      Prof prof(x, TH_K_VECTOR, s);
      if ((st = cuda_status(th::launch_cadd32(uc, x.wc32, x.g.Nc * (long long)nrhs, s))) != TH_OK) return st;
    }
  }
  return st;
}

template <typename T>
th_status coarse_apply_(th_ctx& x, const typename th::Cx<T>::t* in, typename th::Cx<T>::t* out, int nrhs,
                        cudaStream_t s) {
  using B = PrecBufs<T>;
  if (x.gal) {
    const th::GalArgs<T> ga = gal_args<T>(x, in, out, nrhs);
    if (!ga.st) return TH_ERR_UNSUPPORTED;
    x.launches += 1;
    Prof prof(x, TH_K_COARSE_APPLY, s);
    return cuda_status(th::launch_gal_apply<T>(ga, s));
  }
  th::CoarseApplyArgs<T> a{};
  a.x = in;
  a.y = out;
  a.cell = B::cell(x);
  a.rho = B::rho(x);
  a.Nc = x.g.Nc;
  a.nc = x.g.nc;
  a.mc = x.g.mc;
  a.dirichlet = x.g.dirichlet[0] | (x.g.dirichlet[1] << 1) | (x.g.dirichlet[2] << 2) | (x.g.dirichlet[3] << 3);
  x.launches += 1;
  Prof prof(x, TH_K_COARSE_APPLY, s);
  if (x.g.dim == 3) return cuda_status(th::launch_coarse_apply3<T>(a, nrhs, s));
  return cuda_status(th::launch_coarse_apply<T>(a, nrhs, s));
}

// u_c from r_c: the direct coarse solve, the learned corrector or nothing (th_set_coarse)
template <typename T>
th_status coarse_correct_(th_ctx& x, const typename th::Cx<T>::t* rc, typename th::Cx<T>::t* uc, int nrhs,
                          cudaStream_t s) {
  if (x.coarse_mode == 0) return coarse_solve_<T>(x, rc, uc, nrhs, s);
  if (x.coarse_mode == 2) {  // no coarse-grid correction: u_c = 0
    Prof prof(x, TH_K_COARSE_SOLVE, s);
    return cuda_status(cudaMemsetAsync(uc, 0, sizeof(typename th::Cx<T>::t) * x.g.Nc * (size_t)nrhs, s));
  }
  if (!x.unet) return TH_ERR_UNSUPPORTED;
  x.launches += x.unet->launches_per_forward();
  Prof prof(x, TH_K_COARSE_SOLVE, s);
  return cuda_status(x.unet->correct<typename th::Cx<T>::t>(rc, uc, x.g.Nc, nrhs, s));
}

// TwoGridStep(0, f) of Algorithm 1 in precision T (2-D, n_s = n_dd = 1) with
// the vector passes folded into their neighbours, bitwise the same arithmetic
// as the step-by-step form below:
//   V = DD(f);  ua = avg V, r = f - A ua   (one fine apply reading V)
//   r_c = I_P^T r;  u_c = coarse(r_c)
//   ub = ua + omega_c I_P u_c, r = f - A ub   (one fine apply reading u_c)
//   V = DD(r);  out = ub + avg V   (one combine; to `wide` in FP64 if given)
template <typename T>
th_status cycle_fused(th_ctx& x, int wkind, const typename th::Cx<T>::t* f, typename th::Cx<T>::t* u, int nrhs,
                      double2* wide, int wide_acc, cudaStream_t s) {
  using B = PrecBufs<T>;
  using C = typename th::Cx<T>::t;
  const th::Geometry& g = x.g;
  th_status st;
  C* ua = u;
  C* ub = B::s(x);
  if ((st = dd_apply<T>(x, wkind, f, nrhs, s)) != TH_OK) return st;
  // variant 2: every later launch of the step may be scheduled while its
  // predecessor drains (programmatic dependent launch; each kernel waits for
  // it before touching its data); not with per-kernel events or a non-kernel
  // step between two launches
  th::PdlScope pdl(x.fuse == 2 && !x.prof_on && x.coarse_mode == 0);
  auto fused_apply = [&](int src, C* uout) -> th_status {
    th::FineArgs<T> a = fine_args<T>(x, TH_OP_A, nrhs);
    a.u = nullptr;
    a.f = f;
    a.y = B::r(x);
    a.residual = 1;
    a.src = src;
    a.uout = uout;
    a.V = B::V(x);
    a.ctab = x.ctab;
    a.nb = g.nb;
    a.Lu = g.Lu;
    a.NR = g.NR;
    a.nsub = g.nsub;
    a.uin = ua;
    a.uc = B::uc(x);
    a.pj0 = x.pj0;
    a.pw = B::pw(x);
    a.Nc = g.Nc;
    a.mc = g.mc;
    a.q = g.q;
    a.omega = (T)x.prm.omega_c;
    x.launches += 1;
    Prof prof(x, TH_K_FINE, s);
    return cuda_status(th::launch_fine_apply<T>(a, nrhs, s));
  };
  if ((st = fused_apply(1, ua)) != TH_OK) return st;
  if ((st = restrict_<T>(x, B::r(x), B::rc(x), nrhs, s)) != TH_OK) return st;
  if ((st = coarse_correct_<T>(x, B::rc(x), B::uc(x), nrhs, s)) != TH_OK) return st;
  if ((st = fused_apply(2, ub)) != TH_OK) return st;
  if ((st = dd_apply<T>(x, wkind, B::r(x), nrhs, s)) != TH_OK) return st;
  th::CombineArgs<T> a{};
  a.V = B::V(x);
  a.u = u;
  a.uin = ub;
  a.wide = wide;
  a.wide_acc = wide_acc;
  a.ctab = x.ctab;
  a.N = g.N;
  a.m = g.m;
  a.nb = g.nb;
  a.Lu = g.Lu;
  a.NR = g.NR;
  a.nsub = g.nsub;
  x.launches += 1;
  Prof prof(x, TH_K_COMBINE, s);
  return cuda_status(th::launch_dd_combine<T>(a, nrhs, s));
}

template <typename T>
bool can_fuse(const th_ctx& x, bool u_zero) {
  return x.fuse && u_zero && x.g.dim == 2 && x.prm.n_s == 1 && x.prm.n_dd == 1;
}

// TwoGridStep(u, f) of Algorithm 1 in precision T.
template <typename T>
th_status cycle(th_ctx& x, int wkind, const typename th::Cx<T>::t* f, typename th::Cx<T>::t* u, bool u_zero,
                int nrhs, cudaStream_t s) {
  using B = PrecBufs<T>;
  th_status st;
  if (can_fuse<T>(x, u_zero)) return cycle_fused<T>(x, wkind, f, u, nrhs, nullptr, 0, s);
  for (int i = 0; i < x.prm.n_s; ++i)
    if ((st = smooth<T>(x, wkind, f, u, u_zero && i == 0, nrhs, s)) != TH_OK) return st;
  if ((st = fine_apply<T>(x, TH_OP_A, u, f, B::r(x), nrhs, s)) != TH_OK) return st;
  if ((st = restrict_<T>(x, B::r(x), B::rc(x), nrhs, s)) != TH_OK) return st;
  if ((st = coarse_correct_<T>(x, B::rc(x), B::uc(x), nrhs, s)) != TH_OK) return st;
  if ((st = prolong_<T>(x, B::uc(x), u, (T)x.prm.omega_c, nrhs, s)) != TH_OK) return st;
  for (int i = 0; i < x.prm.n_s; ++i)
    if ((st = smooth<T>(x, wkind, f, u, false, nrhs, s)) != TH_OK) return st;
  return TH_OK;
}

// Widen / narrow helpers (interleaved complex = 2 reals per entry)
th_status narrow(th_ctx& x, const double2* in, float2* out, long long n, cudaStream_t s) {
  x.launches += 1;
  Prof prof(x, TH_K_VECTOR, s);
  return cuda_status(th::launch_d2f((const double*)in, (float*)out, 2 * n, s));
}
th_status widen(th_ctx& x, const float2* in, double2* out, long long n, int acc, cudaStream_t s) {
  x.launches += 1;
  Prof prof(x, TH_K_VECTOR, s);
  return cuda_status(th::launch_f2d((const float*)in, (double*)out, 2 * n, acc, s));
}

// z = B v: the two-grid preconditioner (TwoGridStep with u = 0) in the active precision.
// vsplit (mixed forms): v is in the split form of the double-single FGMRES basis.
th_status precondition(th_ctx& x, const double2* v, double2* z, int nrhs, cudaStream_t s, bool vsplit = false) {
  const long long n = x.g.N * (long long)nrhs;
  if (x.active == TH_PREC_FP64) return cycle<double>(x, TH_PREC_FP64, v, z, true, nrhs, s);
  th_status st;
  if (vsplit) {
    x.launches += 1;
    Prof prof(x, TH_K_VECTOR, s);
    if ((st = cuda_status(th::launch_split_to_f32(v, x.f32, n, s))) != TH_OK) return st;
  } else if ((st = narrow(x, v, x.f32, n, s)) != TH_OK) {
    return st;
  }
  if (can_fuse<float>(x, true)) return cycle_fused<float>(x, x.active, x.f32, x.u32, nrhs, z, 0, s);
  if ((st = cycle<float>(x, x.active, x.f32, x.u32, true, nrhs, s)) != TH_OK) return st;
  return widen(x, x.u32, z, n, 0, s);
}

// Runs body(stream) from a CUDA graph: the first call for a key (kind, a, b,
// nrhs, active precision, settings epoch) captures body's launches on the
// private capture stream and instantiates them; every call then launches the
// graph on s, so a cycle costs one host call instead of one per kernel.
constexpr size_t kMaxGraphs = 256;
template <typename F>
th_status graph_run(th_ctx& x, int kind, const void* a, const void* b, int nrhs, cudaStream_t s, F&& body) {
  if (!x.graphs.empty() && x.graphs.front().epoch != x.epoch) x.drop_graphs();  // settings changed
  for (const th_ctx::Graph& gr : x.graphs)
    if (gr.kind == kind && gr.a == a && gr.b == b && gr.nrhs == nrhs && gr.active == x.active &&
        gr.epoch == x.epoch) {
      TH_CU(cudaGraphLaunch(gr.exec, s));
      x.launches += gr.launches;
      return TH_OK;
    }
  if (x.graphs.size() >= kMaxGraphs) x.drop_graphs();
  if (!x.gstream) TH_CU(cudaStreamCreateWithFlags(&x.gstream, cudaStreamNonBlocking));
  const long long l0 = x.launches;
  TH_CU(cudaStreamBeginCapture(x.gstream, cudaStreamCaptureModeThreadLocal));
  const th_status st = body(x.gstream);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(x.gstream, &graph);
  const long long nl = x.launches - l0;
  x.launches = l0;  // nothing ran during the capture
  if (st != TH_OK || ce != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return st != TH_OK ? st : TH_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return TH_ERR_CUDA;
  x.graphs.push_back({kind, nrhs, x.active, a, b, x.epoch, nl, exec});
  TH_CU(cudaGraphLaunch(exec, s));
  x.launches += nl;
  return TH_OK;
}

th_status check_nrhs(const th_ctx* x, int nrhs) {
  if (!x) return TH_ERR_ARG;
  if (nrhs < 1 || nrhs > x->prm.nrhs_max) return TH_ERR_ARG;
  return TH_OK;
}

th_status norms(th_ctx& x, const double2* w, int nrhs, std::vector<double>& out, cudaStream_t s) {
  x.launches += 2;
  {
    Prof prof(x, TH_K_KRYLOV, s);
    TH_CU(th::launch_norm2(w, x.g.N, nrhs, x.npart, x.nrm, x.nblk, s));
  }
  out.resize(nrhs);
  TH_CU(cudaMemcpyAsync(out.data(), x.nrm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  TH_CU(cudaStreamSynchronize(s));
  for (auto& v : out) v = std::sqrt(v);
  return TH_OK;
}

}  // namespace

namespace {
// Set-up autotuner: times the fine-apply tile variants on this problem with
// CUDA events, for nrhs right-hand sides, and keeps the faster one (T = ds:
// the double-single apply, FP64 input and FP32 output).
template <typename T>
th_status tune_fine(th_ctx& x, cudaStream_t s, int nrhs, int& choice) {
  using C = typename th::Cx<T>::t;
  C* u = nullptr;
  C* y = nullptr;
  size_t ubytes = 0;
  if constexpr (std::is_same<T, double>::value) {
    u = x.r64;
    y = x.t64;
    ubytes = sizeof(double2);
  } else if constexpr (std::is_same<T, th::ds>::value) {
    u = reinterpret_cast<C*>(x.r64);
    y = reinterpret_cast<C*>(x.r32);
    ubytes = sizeof(double2);
    if (!x.kcds) return TH_OK;
  } else {
    u = x.f32;
    y = x.r32;
    ubytes = sizeof(float2);
  }
  if (!u || !y) return TH_OK;
  TH_CU(cudaMemsetAsync(u, 0, ubytes * x.g.N * (size_t)nrhs, s));
  cudaEvent_t e0, e1;
  TH_CU(cudaEventCreate(&e0));
  TH_CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int arg = 0;
  for (int v = 0; v < 2; ++v) {
    th::FineArgs<T> a = fine_args<T>(x, TH_OP_A, 1);
    a.tc = v;
    a.u = u;
    a.y = y;
    a.f = nullptr;
    a.residual = 0;
    for (int w = 0; w < 2; ++w) TH_CU(th::launch_fine_apply<T>(a, nrhs, s));
    TH_CU(cudaEventRecord(e0, s));
    for (int r = 0; r < 5; ++r) TH_CU(th::launch_fine_apply<T>(a, nrhs, s));
    TH_CU(cudaEventRecord(e1, s));
    TH_CU(cudaEventSynchronize(e1));
    float ms = 0;
    TH_CU(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) { best = ms; arg = v; }
  }
  choice = arg;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return TH_OK;
}

// times the two one-rhs coarse sweeps (precision T) and keeps the faster
template <typename T>
th_status tune_coarse(th_ctx& x, cudaStream_t s, int& choice) {
  using C = typename th::Cx<T>::t;
  C *rc = nullptr, *uc = nullptr;
  if constexpr (std::is_same<T, double>::value) {
    rc = x.rc64;
    uc = x.uc64;
  } else {
    rc = x.rc32;
    uc = x.uc32;
  }
  if (!rc || !uc || x.g.dim != 2) return TH_OK;
  TH_CU(cudaMemsetAsync(rc, 0, sizeof(C) * x.g.Nc, s));
  cudaEvent_t e0, e1;
  TH_CU(cudaEventCreate(&e0));
  TH_CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int arg = choice;
  for (int v = 0; v < 3; ++v) {
    choice = v;
    bool ok = true;
    for (int w = 0; w < 2 && ok; ++w) ok = (coarse_solve_<T>(x, rc, uc, 1, s) == TH_OK);
    if (!ok) {
      cudaGetLastError();
      continue;
    }
    TH_CU(cudaEventRecord(e0, s));
    for (int k = 0; k < 4; ++k)
      if (coarse_solve_<T>(x, rc, uc, 1, s) != TH_OK) ok = false;
    TH_CU(cudaEventRecord(e1, s));
    TH_CU(cudaEventSynchronize(e1));
    float ms = 0;
    TH_CU(cudaEventElapsedTime(&ms, e0, e1));
    if (ok && ms < best) { best = ms; arg = v; }
  }
  choice = arg;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return TH_OK;
}

// Accuracy check of the mixed form's 2-D coarse solve: on seeded right-hand
// sides (1 and, with nrhs_max >= 8, 8 of them: the grouped path), refinement
// steps are added, at most 2, while the FP32 coarse residual
// max_i ||r_i - A_q u_i|| / ||r_i|| exceeds 1e-3.  On large coarse grids the
// partitioned FP32 solve loses several digits (its chunk systems amplify the
// rounding errors) and the outer iteration then needs more steps; one
// refinement step restores the FP64 solve's accuracy to about 1e-5.
th_status tune_coarse_refine(th_ctx& x, cudaStream_t s) {
  x.coarse_refine = 0;
  if (!x.zc32 || !x.wc32 || !x.rc32 || !x.uc32 || x.g.dim != 2 || x.gal) return TH_OK;
  const long long Nc = x.g.Nc;
  const int nmax = x.prm.nrhs_max >= 8 ? 8 : 1;
  std::vector<float2> h((size_t)nmax * Nc), z(h.size());
  uint64_t st = 0x2545F4914F6CDD1Dull;  // xorshift64, values uniform in [-1, 1)
  auto next = [&]() {
    st ^= st << 13;
    st ^= st >> 7;
    st ^= st << 17;
    return (float)((double)(st >> 11) * (2.0 / 9007199254740992.0) - 1.0);
  };
  for (float2& v : h) {
    v.x = next();
    v.y = next();
  }
  TH_CU(cudaMemcpyAsync(x.rc32, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
  TH_CU(cudaStreamSynchronize(s));
  int need = 0;
  for (int nrhs : {1, nmax}) {
    for (int r = 0; r <= 2; ++r) {
      x.coarse_refine = r;
      th_status e = coarse_solve_<float>(x, x.rc32, x.uc32, nrhs, s);
      if (e == TH_OK) e = coarse_residual32(x, x.rc32, x.uc32, x.zc32, nrhs, s);
      if (e != TH_OK) return e;
      TH_CU(cudaMemcpyAsync(z.data(), x.zc32, (size_t)nrhs * Nc * sizeof(float2), cudaMemcpyDeviceToHost, s));
      TH_CU(cudaStreamSynchronize(s));
      double worst = 0.0;
      for (int i = 0; i < nrhs; ++i) {
        double zz = 0.0, rr = 0.0;
        for (long long j = 0; j < Nc; ++j) {
          const float2 a = z[(size_t)i * Nc + j], b = h[(size_t)i * Nc + j];
          zz += (double)a.x * a.x + (double)a.y * a.y;
          rr += (double)b.x * b.x + (double)b.y * b.y;
        }
        worst = std::max(worst, std::sqrt(zz / rr));
      }
      if (!(worst > 1e-3) || r == 2) {
        need = std::max(need, r);
        break;
      }
    }
  }
  x.coarse_refine = need;
  return TH_OK;
}

template <typename T>
th_status tune_dd(th_ctx& x, int wkind, cudaStream_t s, int& choice) {
  using C = typename th::Cx<T>::t;
  C* r = nullptr;
  if constexpr (std::is_same<T, double>::value) r = x.r64; else r = x.r32;
  if (!r || !x.W[wkind]) return TH_OK;
  // timed at the batch width the context was set up for (up to 8 right-hand sides):
  // the best variant for one rhs is not the best for tiles of several
  const int nt = std::max(1, std::min(x.prm.nrhs_max, 8));
  TH_CU(cudaMemsetAsync(r, 0, sizeof(C) * x.g.N * nt, s));
  // the CUDA-core variants are compared (the tensor-core path does not depend on them)
  const int saved_tc = x.dd_tc;
  x.dd_tc = 0;
  struct TcRestore {
    th_ctx& x;
    int v;
    ~TcRestore() { x.dd_tc = v; }
  } tc_restore{x, saved_tc};
  cudaEvent_t e0, e1;
  TH_CU(cudaEventCreate(&e0));
  TH_CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int arg = 0;
  // 4 and 5 (paired FP32 FMAs) exist for FP32 arithmetic on BF16 / FP16 rows only
  const int nv = (std::is_same<T, float>::value && (wkind == TH_PREC_BF16 || wkind == TH_PREC_FP16)) ? 6 : 4;
  for (int v = 0; v < nv; ++v) {
    choice = v;
    bool ok = true;
    for (int w = 0; w < 2 && ok; ++w) ok = (dd_apply<T>(x, wkind, r, nt, s) == TH_OK);
    if (!ok) {
      cudaGetLastError();
      continue;
    }
    TH_CU(cudaEventRecord(e0, s));
    for (int k = 0; k < 4; ++k)
      if (dd_apply<T>(x, wkind, r, nt, s) != TH_OK) ok = false;
    TH_CU(cudaEventRecord(e1, s));
    TH_CU(cudaEventSynchronize(e1));
    float ms = 0;
    TH_CU(cudaEventElapsedTime(&ms, e0, e1));
    if (ok && ms < best) { best = ms; arg = v; }
  }
  choice = arg;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return TH_OK;
}

}  // namespace

namespace th {
// Read-only view of the FP64 coarse factors of a context (for th_coarse_solve_noalloc).
bool coarse_factors_fp64(const th_ctx* x, CoarseSolveArgs<double>* a, int* cluster, int* nrhs_max, int* device) {
  if (!x || !x->G64) return false;
  *device = x->device;
  a->G = x->G64;
  a->cl = x->cl64;
  a->cd = x->cd64;
  a->cu = x->cu64;
  a->Nc = x->g.Nc;
  a->mc = x->g.mc;
  a->rpc = x->rpc;
  *cluster = x->cluster;
  *nrhs_max = x->prm.nrhs_max;
  return true;
}
}  // namespace th

// ====================================================================== ABI
extern "C" {

const char* th_status_str(th_status s) {
  switch (s) {
    case TH_OK: return "ok";
    case TH_ERR_ARG: return "invalid argument";
    case TH_ERR_CUDA: return "CUDA error";
    case TH_ERR_NOMEM: return "workspace too small or host allocation failed";
    case TH_ERR_NOCONV: return "not converged within maxit";
    case TH_ERR_BREAKDOWN: return "Krylov breakdown";
    case TH_ERR_NONFINITE: return "non-finite value in a residual norm";
    case TH_ERR_TIMEOUT: return "device wait timed out";
    case TH_ERR_UNSUPPORTED: return "unsupported configuration";
    case TH_ERR_SINGULAR: return "singular matrix in set-up";
  }
  return "unknown status";
}

th_status th_workspace_size(const th_mesh* mesh, const th_params* prm, size_t* bytes) {
  if (!bytes) return TH_ERR_ARG;
  th_ctx x;
  th_status st = prepare(mesh, prm, x);
  if (st != TH_OK) return st;
  Carve c;
  carve_all(x, c);
  *bytes = c.used + 256;
  return TH_OK;
}

th_status th_setup(const th_mesh* mesh, const double* k_host, const double* eps_host, const th_params* prm,
                   void* workspace_dev, size_t bytes, void* stream, th_ctx** out) {
  if (!out || !k_host || !workspace_dev) return TH_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<th_ctx> x(new (std::nothrow) th_ctx());
  if (!x) return TH_ERR_NOMEM;
  th_status st = prepare(mesh, prm, *x);
  if (st != TH_OK) return st;
  const th::Geometry& g = x->g;
  const bool d3 = g.dim == 3;
  const size_t n2 = (size_t)g.n * g.n * (d3 ? g.n : 1);  // cells
  x->k_host.assign(k_host, k_host + n2);
  for (size_t i = 0; i < n2; ++i) {
    if (!std::isfinite(k_host[i]) || k_host[i] <= 0.0) return TH_ERR_ARG;
    if (eps_host && (!std::isfinite(eps_host[i]) || eps_host[i] < 0.0)) return TH_ERR_ARG;
  }
  Carve c;
  c.base = reinterpret_cast<char*>(workspace_dev);
  c.cap = bytes;
  if ((reinterpret_cast<uintptr_t>(workspace_dev) & 255u) != 0) return TH_ERR_ARG;
  carve_all(*x, c);
  if (!c.ok) return TH_ERR_NOMEM;
  cudaStream_t s = S(stream);
  std::vector<double> eps0;
  const double* eps = eps_host;
  if (!eps) {
    eps0.assign(n2, 0.0);
    eps = eps0.data();
  }

  // --- host FP64 set-up
  th::TransferTables tt;
  th::transfer_tables(g, x->ref, tt);
  th::CoarseBlocks cb;
  th::CoarsePart cpart;
  th::CoarseBlocks3 cb3;
  th::GalBlocks gb;
  const bool qs2 = !d3 && !x->gal;  // 2-D QSFEM coarse level
  if (x->gal) {
    if ((st = th::galerkin_setup(g, k_host, eps, x->prm.alpha_c, gb)) != TH_OK) return st;
  } else if (!d3) {
    // the unpartitioned block inverses only for the FP64 no-alloc sweep
    if ((st = th::coarse_setup(g, k_host, eps, cb, x->G64 != nullptr)) != TH_OK) return st;
    if ((st = th::coarse_partition(g, cb, x->P, cpart)) != TH_OK) return st;
  } else {
    if ((st = th::coarse_setup3(g, k_host, eps, cb3)) != TH_OK) return st;
  }
  std::vector<cplx> Wh;
  if ((st = th::all_inverse_rows(g, x->ref, k_host, eps, x->prm.alpha_s, Wh)) != TH_OK) return st;

  // --- uploads (synchronous copies from host vectors)
  auto up = [&](void* dst, const void* src, size_t nb) -> th_status {
    if (!dst || nb == 0) return TH_OK;
    return cuda_status(cudaMemcpyAsync(dst, src, nb, cudaMemcpyHostToDevice, s));
  };
  std::vector<int4> ctab(g.m);
  for (int i = 0; i < g.m; ++i)
    ctab[i] = make_int4(g.ctab[i * 4], g.ctab[i * 4 + 1], g.ctab[i * 4 + 2], g.ctab[i * 4 + 3]);
  std::vector<float> kf(n2), ef(n2), pwf(tt.pw.size()), rwf(tt.rw.size());
  for (size_t i = 0; i < n2; ++i) { kf[i] = (float)k_host[i]; ef[i] = (float)eps[i]; }
  for (size_t i = 0; i < tt.pw.size(); ++i) pwf[i] = (float)tt.pw[i];
  for (size_t i = 0; i < tt.rw.size(); ++i) rwf[i] = (float)tt.rw[i];
  std::vector<double2> rho64;
  if (qs2) {
    rho64.resize(4 * (size_t)g.nc);
    for (int sd = 0; sd < 4; ++sd)
      for (int t = 0; t < g.nc; ++t) rho64[(size_t)sd * g.nc + t] = make_double2(cb.rho[sd][t].real(), cb.rho[sd][t].imag());
  } else if (d3) {
    rho64.resize(cb3.rho.size());
    for (size_t i = 0; i < cb3.rho.size(); ++i) rho64[i] = make_double2(cb3.rho[i].real(), cb3.rho[i].imag());
  }
  const size_t mm = (size_t)g.mc * g.mc;
  auto to2 = [](const std::vector<cplx>& v) {
    std::vector<double2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = make_double2(v[i].real(), v[i].imag());
    return o;
  };
  auto to2f = [](const std::vector<cplx>& v) {
    std::vector<float2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].real(), (float)v[i].imag());
    return o;
  };
  std::vector<double2> cell64 = to2(d3 ? cb3.cell : cb.cell), cl64 = to2(cb.cl), cd64 = to2(cb.cd),
                       cu64 = to2(cb.cu);
  if ((st = up(x->kc64, k_host, n2 * 8)) != TH_OK) return st;
  if ((st = up(x->ec64, eps, n2 * 8)) != TH_OK) return st;
  if ((st = up(x->box, g.box.data(), g.box.size() * 4)) != TH_OK) return st;
  if ((st = up(x->ctab, ctab.data(), ctab.size() * sizeof(int4))) != TH_OK) return st;
  if ((st = up(x->pj0, tt.pj0.data(), tt.pj0.size() * 4)) != TH_OK) return st;
  if ((st = up(x->pw64, tt.pw.data(), tt.pw.size() * 8)) != TH_OK) return st;
  if ((st = up(x->ridx, tt.ridx.data(), tt.ridx.size() * 4)) != TH_OK) return st;
  if ((st = up(x->rw64, tt.rw.data(), tt.rw.size() * 8)) != TH_OK) return st;
  if ((st = up(x->ccell64, cell64.data(), cell64.size() * 16)) != TH_OK) return st;
  if ((st = up(x->crho64, rho64.data(), rho64.size() * 16)) != TH_OK) return st;
  if (qs2) {
    if ((st = up(x->cl64, cl64.data(), mm * 16)) != TH_OK) return st;
    if ((st = up(x->cd64, cd64.data(), mm * 16)) != TH_OK) return st;
    if ((st = up(x->cu64, cu64.data(), mm * 16)) != TH_OK) return st;
  }
  std::vector<double2> G64h;
  if (x->G64) {
    G64h = to2(cb.G);
    if ((st = up(x->G64, G64h.data(), G64h.size() * 16)) != TH_OK) return st;
  }
  if (qs2) {
    std::vector<int> chunk_of(g.mc, -1);
    for (int c = 0; c < x->P; ++c)
      for (int j = cpart.ca[c]; j <= cpart.cb[c]; ++j) chunk_of[j] = c;
    std::vector<int> sep(std::max(x->P - 1, 1), 0);
    std::copy(cpart.sep.begin(), cpart.sep.end(), sep.begin());
    if ((st = up(x->ca, cpart.ca.data(), cpart.ca.size() * 4)) != TH_OK) return st;
    if ((st = up(x->cb, cpart.cb.data(), cpart.cb.size() * 4)) != TH_OK) return st;
    if ((st = up(x->sep, sep.data(), sep.size() * 4)) != TH_OK) return st;
    if ((st = up(x->chunk_of, chunk_of.data(), chunk_of.size() * 4)) != TH_OK) return st;
    TH_CU(cudaStreamSynchronize(s));
  }
  // partitioned factors, FP64 and/or FP32 (one staging vector at a time)
  auto upload_c = [&](double2* d64, float2* d32, const std::vector<cplx>& v) -> th_status {
    if (d64) {
      std::vector<double2> t = to2(v);
      th_status r = up(d64, t.data(), t.size() * 16);
      if (r != TH_OK) return r;
      if (cudaStreamSynchronize(s) != cudaSuccess) return TH_ERR_CUDA;
    }
    if (d32) {
      std::vector<float2> t = to2f(v);
      th_status r = up(d32, t.data(), t.size() * 8);
      if (r != TH_OK) return r;
      if (cudaStreamSynchronize(s) != cudaSuccess) return TH_ERR_CUDA;
    }
    return TH_OK;
  };
  if (d3) {
    if ((st = upload_c(x->G3_64, x->G3_32, cb3.G)) != TH_OK) return st;
    if ((st = upload_c(x->dn64, x->dn32, cb3.dn)) != TH_OK) return st;
    if ((st = upload_c(x->up64, x->up32, cb3.up)) != TH_OK) return st;
  }
  if (x->gal) {
    if ((st = upload_c(x->gst64, x->gst32, gb.st)) != TH_OK) return st;
    if ((st = upload_c(x->gG64, x->gG32, gb.G)) != TH_OK) return st;
    std::vector<cplx>().swap(gb.G);
  }
  if ((st = upload_c(x->Gp64, x->Gp32, cpart.G)) != TH_OK) return st;
  if (x->Gt64 || x->Gt32) {
    // G_j^T with rows padded to mcr: Gt[j][c][row] = G[j][row][c]
    const size_t mcr = (size_t)x->mcr, mcp = (size_t)x->mcp;
    std::vector<cplx> gt((size_t)g.mc * g.mc * mcr, cplx(0.0));
    th::parallel_for(g.mc, [&](int j) {
      for (int row = 0; row < g.mc; ++row)
        for (int c = 0; c < g.mc; ++c)
          gt[((size_t)j * g.mc + c) * mcr + row] = cpart.G[((size_t)j * g.mc + row) * mcp + c];
    });
    if ((st = upload_c(x->Gt64, x->Gt32, gt)) != TH_OK) return st;
  }
  if ((st = upload_c(x->LR64, x->LR32, cpart.LR)) != TH_OK) return st;
  if (x->LRt32) {
    // LRt[j][col][row] = LR[j][row][col], rows padded to mcr
    const size_t mcr = (size_t)x->mcr, K = 2 * (size_t)x->mcp;
    std::vector<cplx> lt((size_t)g.mc * K * mcr, cplx(0.0));
    th::parallel_for(g.mc, [&](int j) {
      for (int row = 0; row < g.mc; ++row)
        for (size_t c = 0; c < K; ++c) lt[((size_t)j * K + c) * mcr + row] = cpart.LR[((size_t)j * g.mc + row) * K + c];
    });
    if ((st = upload_c(nullptr, x->LRt32, lt)) != TH_OK) return st;
  }
  if (x->Sb16 && x->LRb16) {
    // split-BF16 operands of the tensor-core separator product and spike
    // correction: 128-row tiles, 32-column chunks of four parts (re hi, im hi,
    // re lo, im lo; v = hi + lo, hi = bf16(v), lo = bf16(v - hi)) in the K-major
    // core-matrix layout (umma_off32); padding rows and columns are zero
    const int mc = g.mc, nred = x->nred, nkc_s = x->nkc_s, nkc_m = x->nkc_m;
    const size_t K = 2 * (size_t)x->mcp;  // row length of cpart.LR
    std::vector<th::CoarseTile> ts, tl;
    {
      std::vector<uint16_t> sb((size_t)x->ntiles_s * nkc_s * 16384, 0);
      th::parallel_for(x->ntiles_s, [&](int t) {
        for (int kc = 0; kc < nkc_s; ++kc) {
          uint16_t* ch = sb.data() + ((size_t)t * nkc_s + kc) * 16384;
          for (int r = 0; r < 128; ++r) {
            const int row = t * 128 + r;
            if (row >= nred) break;
            for (int k = 0; k < 32; ++k) {
              const int col = kc * 32 + k;
              if (col >= nred) break;
              put_split(ch, th::umma_off32(r, k), 4096, cpart.Sinv[(size_t)row * nred + col]);
            }
          }
        }
      });
      // per tile and K split: the split's first chunk (b0) and index (b1)
      const int ns = x->nsplit_s;
      for (int t = 0; t < x->ntiles_s; ++t)
        for (int sp = 0; sp < ns; ++sp) {
          const int k0 = (int)((long long)sp * nkc_s / ns), k1 = (int)((long long)(sp + 1) * nkc_s / ns);
          ts.push_back(th::CoarseTile{((long long)t * nkc_s + k0) * 32768, k1 - k0, t * 128,
                                      std::min(128, nred - t * 128), k0, sp});
        }
      if ((st = up(x->Sb16, sb.data(), sb.size() * 2)) != TH_OK) return st;
      TH_CU(cudaStreamSynchronize(s));
    }
    {
      long long chunk0 = 0;
      std::vector<int> tch;  // chunk of each tile
      for (int ch = 0; ch < x->P; ++ch) {
        const int L = cpart.cb[ch] - cpart.ca[ch] + 1, nrow = L * mc;
        // separators: chunk 0 has only its right one (index 0), the last chunk only its left one
        const int b0 = ch > 0 ? ch - 1 : ch, b1 = (ch > 0 && ch < x->P - 1) ? ch : -1;
        const int nkc = (b1 >= 0 ? 2 : 1) * nkc_m;
        for (int r0 = 0; r0 < nrow; r0 += 128) {
          tl.push_back(th::CoarseTile{chunk0 * 32768, nkc, cpart.ca[ch] * mc + r0, std::min(128, nrow - r0), b0, b1});
          tch.push_back(ch);
          chunk0 += nkc;
        }
      }
      if ((int)tl.size() != x->ntiles_l || chunk0 != x->lrb_chunks) return TH_ERR_ARG;  // partition mismatch
      std::vector<uint16_t> lb((size_t)x->lrb_chunks * 16384, 0);
      th::parallel_for(x->ntiles_l, [&](int t) {
        const th::CoarseTile& tt = tl[t];
        for (int kc = 0; kc < tt.nkc; ++kc) {
          // column block of [L | R]: 0 = the left separator's coupling, 1 = the right one's
          const int side = tt.b1 >= 0 ? kc / nkc_m : (tch[t] == 0 ? 1 : 0);
          uint16_t* chp = lb.data() + ((size_t)(tt.a_off / 32768) + kc) * 16384;
          for (int r = 0; r < tt.rows; ++r) {
            const size_t xi = (size_t)tt.row0 + r;  // coarse index: block row j, entry rr
            const size_t j = xi / mc, rr = xi % mc;
            for (int k = 0; k < 32; ++k) {
              const int col = (kc % nkc_m) * 32 + k;
              if (col >= mc) break;
              put_split(chp, th::umma_off32(r, k), 4096, cpart.LR[(j * mc + rr) * K + (size_t)side * x->mcp + col]);
            }
          }
        }
      });
      if ((st = up(x->LRb16, lb.data(), lb.size() * 2)) != TH_OK) return st;
      if ((st = up(x->tiles_s, ts.data(), ts.size() * sizeof(th::CoarseTile))) != TH_OK) return st;
      if ((st = up(x->tiles_l, tl.data(), tl.size() * sizeof(th::CoarseTile))) != TH_OK) return st;
      TH_CU(cudaStreamSynchronize(s));
    }
    const size_t groups = (size_t)(x->prm.nrhs_max + 63) / 64;
    TH_CU(cudaMemsetAsync(x->rst16, 0, groups * nkc_s * 16384, s));
    TH_CU(cudaMemsetAsync(x->xst16, 0, groups * (x->P - 1) * nkc_m * 16384, s));
    th::CoarseUmmaArgs& u = x->umma;
    u.As = x->Sb16;
    u.Al = x->LRb16;
    u.tiles_s = x->tiles_s;
    u.tiles_l = x->tiles_l;
    u.ntiles_s = x->ntiles_s * x->nsplit_s;
    u.nsplit = x->nsplit_s;
    u.spart = x->spart_s;
    u.nrhs_cap = (int)groups * 64;
    u.nred = nred;
    u.ntiles_l = x->ntiles_l;
    u.rst = x->rst16;
    u.xst = x->xst16;
    u.sep = x->sep;
    u.Nc = g.Nc;
    u.mc = mc;
    u.nsep = x->P - 1;
    u.nkc_s = nkc_s;
    u.nkc_m = nkc_m;
  }
  if (x->P > 1 && (x->Si64 || x->Si32)) {
    // rows padded to an even length (pairs of complex values per load)
    const size_t nr_ = (size_t)x->nred, ld = nr_ + (nr_ & 1);
    std::vector<cplx> sp(nr_ * ld, cplx(0.0));
    for (size_t r = 0; r < nr_; ++r) std::copy(&cpart.Sinv[r * nr_], &cpart.Sinv[r * nr_] + nr_, &sp[r * ld]);
    if ((st = upload_c(x->Si64, x->Si32, sp)) != TH_OK) return st;
  }
  if (x->Ssym32 && x->sym_ij) {
    // Sinv's upper-triangle 64 x 64 blocks (I <= J), row-major, zero padded
    const int T = x->Tsym, nred = x->nred;
    std::vector<int2> ij;
    for (int I = 0; I < T; ++I)
      for (int J = I; J < T; ++J) ij.push_back(make_int2(I, J));
    if ((int)ij.size() != x->nsym) return TH_ERR_ARG;
    std::vector<float2> sb((size_t)x->nsym * 64 * 64, make_float2(0.f, 0.f));
    th::parallel_for(x->nsym, [&](int b) {
      const int I = ij[b].x, J = ij[b].y;
      for (int r = 0; r < 64; ++r) {
        const int row = I * 64 + r;
        if (row >= nred) break;
        for (int c = 0; c < 64; ++c) {
          const int col = J * 64 + c;
          if (col >= nred) break;
          const cplx v = cpart.Sinv[(size_t)row * nred + col];
          sb[((size_t)b * 64 + r) * 64 + c] = make_float2((float)v.real(), (float)v.imag());
        }
      }
    });
    if ((st = up(x->Ssym32, sb.data(), sb.size() * sizeof(float2))) != TH_OK) return st;
    if ((st = up(x->sym_ij, ij.data(), ij.size() * sizeof(int2))) != TH_OK) return st;
    TH_CU(cudaStreamSynchronize(s));
  }
  std::vector<float2> cell32, rho32, cl32, cd32, cu32;
  if (x->mixed) {
    cell32 = to2f(d3 ? cb3.cell : cb.cell);
    cl32 = to2f(cb.cl);
    cd32 = to2f(cb.cd);
    cu32 = to2f(cb.cu);
    rho32.resize(rho64.size());
    for (size_t i = 0; i < rho64.size(); ++i) rho32[i] = make_float2((float)rho64[i].x, (float)rho64[i].y);
    if ((st = up(x->kc32, kf.data(), n2 * 4)) != TH_OK) return st;
    if ((st = up(x->ec32, ef.data(), n2 * 4)) != TH_OK) return st;
    if (x->kcds) {
      std::vector<th::ds> kd(n2), ed(n2);
      for (size_t i = 0; i < n2; ++i) {
        kd[i] = th::ds_from_host(k_host[i]);
        ed[i] = th::ds_from_host(eps[i]);
      }
      if ((st = up(x->kcds, kd.data(), n2 * sizeof(th::ds))) != TH_OK) return st;
      if ((st = up(x->ecds, ed.data(), n2 * sizeof(th::ds))) != TH_OK) return st;
      TH_CU(cudaStreamSynchronize(s));
    }
    if ((st = up(x->pw32, pwf.data(), pwf.size() * 4)) != TH_OK) return st;
    if ((st = up(x->rw32, rwf.data(), rwf.size() * 4)) != TH_OK) return st;
    if ((st = up(x->ccell32, cell32.data(), cell32.size() * 8)) != TH_OK) return st;
    if ((st = up(x->crho32, rho32.data(), rho32.size() * 8)) != TH_OK) return st;
    if (qs2) {
      if ((st = up(x->cl32, cl32.data(), mm * 8)) != TH_OK) return st;
      if ((st = up(x->cd32, cd32.data(), mm * 8)) != TH_OK) return st;
      if ((st = up(x->cu32, cu32.data(), mm * 8)) != TH_OK) return st;
    }
  }
  // inverse rows in the chunk-major layouts
  const size_t blk = (size_t)g.NR * g.NC;
  std::vector<uint4> stage;
  std::vector<float> scale16;
  for (int kind = 0; kind < 4; ++kind) {
    if (!x->W[kind]) continue;
    const int NCH = x->wchunks[kind];
    stage.assign((size_t)g.nsub * NCH * g.NR, make_uint4(0, 0, 0, 0));
    if (kind == TH_PREC_FP16) scale16.assign(g.nsub, 1.0f);
    th::parallel_for(g.nsub, [&](int sub) {
      const cplx* src = Wh.data() + blk * sub;
      float sc = 1.0f;
      if (kind == TH_PREC_FP16) {
        double mx = 0.0;
        for (size_t i = 0; i < blk; ++i) mx = std::max(mx, std::max(std::fabs(src[i].real()), std::fabs(src[i].imag())));
        sc = mx > 0 ? (float)(mx / 4096.0) : 1.0f;
        scale16[sub] = sc;
      }
      for (int ch = 0; ch < NCH; ++ch)
        for (int r = 0; r < g.NR; ++r) {
          uint4& o = stage[((size_t)sub * NCH + ch) * g.NR + r];
          if (kind == TH_PREC_FP64) {
            const cplx v = src[(size_t)r * g.NC + ch];
            double2 d = make_double2(v.real(), v.imag());
            std::memcpy(&o, &d, 16);
          } else if (kind == TH_PREC_FP32) {
            float f[4] = {0, 0, 0, 0};
            for (int j = 0; j < 2; ++j) {
              const int c = ch * 2 + j;
              if (c < g.NC) {
                f[2 * j] = (float)src[(size_t)r * g.NC + c].real();
                f[2 * j + 1] = (float)src[(size_t)r * g.NC + c].imag();
              }
            }
            std::memcpy(&o, f, 16);
          } else {
            uint32_t wv[4] = {0, 0, 0, 0};
            for (int j = 0; j < 4; ++j) {
              const int c = ch * 4 + j;
              if (c >= g.NC) continue;
              const cplx v = src[(size_t)r * g.NC + c];
              if (kind == TH_PREC_BF16) {
                wv[j] = (uint32_t)f2bf((float)v.real()) | ((uint32_t)f2bf((float)v.imag()) << 16);
              } else {
                __half hr = __float2half_rn((float)(v.real() / sc));
                __half hi = __float2half_rn((float)(v.imag() / sc));
                uint16_t a, b;
                std::memcpy(&a, &hr, 2);
                std::memcpy(&b, &hi, 2);
                wv[j] = (uint32_t)a | ((uint32_t)b << 16);
              }
            }
            std::memcpy(&o, wv, 16);
          }
        }
    });
    if ((st = up(x->W[kind], stage.data(), stage.size() * 16)) != TH_OK) return st;
    if (kind == TH_PREC_FP16 && (st = up(x->wscale16, scale16.data(), scale16.size() * 4)) != TH_OK) return st;
    // copies read host memory asynchronously: finish before the staging buffer is reused
    TH_CU(cudaStreamSynchronize(s));
  }
  if (x->Wu) {
    // per subdomain: K-chunks of 64 columns, each [re | im] x [row/8][k/8 in chunk][8 rows][8 columns] BF16
    const int M8 = (g.NR + 7) / 8, K8 = 2 * ((g.NC + 15) / 16);
    const size_t sub_bytes = th::dd_umma_bytes_per_sub(g.NR, g.NC);
    std::vector<uint16_t> ustage(sub_bytes / 2 * (size_t)g.nsub, 0);
    th::parallel_for(g.nsub, [&](int sub) {
      const cplx* src = Wh.data() + blk * sub;
      uint16_t* base = ustage.data() + (size_t)sub * sub_bytes / 2;
      for (int kc = 0; kc * 8 < K8; ++kc) {
        const int kcs = std::min(8, K8 - kc * 8);
        uint16_t* chunk = base + (size_t)kc * 8 * 2 * M8 * 64;
        for (int ri = 0; ri < 2; ++ri) {
          uint16_t* part = chunk + (size_t)ri * M8 * kcs * 64;
          for (int mrow = 0; mrow < M8 * 8; ++mrow)
            for (int k8 = 0; k8 < kcs; ++k8)
              for (int e = 0; e < 8; ++e) {
                const int col = (kc * 8 + k8) * 8 + e;
                double v = 0.0;
                if (mrow < g.NR && col < g.NC) {
                  const cplx w = src[(size_t)mrow * g.NC + col];
                  v = ri ? w.imag() : w.real();
                }
                part[((size_t)(mrow / 8) * kcs + k8) * 64 + (mrow % 8) * 8 + e] = f2bf((float)v);
              }
        }
      }
    });
    if ((st = up(x->Wu, ustage.data(), ustage.size() * 2)) != TH_OK) return st;
    TH_CU(cudaStreamSynchronize(s));
  }
  TH_CU(cudaStreamSynchronize(s));
  {
    int dev = 0;
    TH_CU(cudaGetDevice(&dev));
    x->device = dev;
    TH_CU(cudaDeviceGetAttribute(&x->sms, cudaDevAttrMultiProcessorCount, dev));
    TH_CU(cudaMemsetAsync(x->derr, 0, 64 * sizeof(int), s));
  }
  if (!d3) {  // the 3-D apply has one variant
    const int nm = x->prm.nrhs_max;
    if ((st = tune_fine<double>(*x, s, 1, x->tc64)) != TH_OK) return st;
    x->tc64m = x->tc64;
    if (nm >= 8 && (st = tune_fine<double>(*x, s, nm, x->tc64m)) != TH_OK) return st;
    if (x->mixed) {
      if ((st = tune_fine<float>(*x, s, 1, x->tc32)) != TH_OK) return st;
      if ((st = tune_fine<th::ds>(*x, s, 1, x->tcds)) != TH_OK) return st;
      x->tc32m = x->tc32;
      x->tcdsm = x->tcds;
      if (nm >= 8 && (st = tune_fine<float>(*x, s, nm, x->tc32m)) != TH_OK) return st;
      if (nm >= 8 && (st = tune_fine<th::ds>(*x, s, nm, x->tcdsm)) != TH_OK) return st;
    }
  }
  if (x->W[TH_PREC_FP64] && (st = tune_dd<double>(*x, TH_PREC_FP64, s, x->dds64)) != TH_OK) return st;
  if (x->mixed) {
    const int wk = (x->active != TH_PREC_FP64) ? x->active : (x->W[TH_PREC_BF16] ? TH_PREC_BF16 : TH_PREC_FP32);
    if (x->W[wk] && (st = tune_dd<float>(*x, wk, s, x->dds32)) != TH_OK) return st;
  }
  if (qs2) {
    // one sweep variant serves both precisions: time it where the cycle runs
    if (x->mixed) {
      if ((st = tune_coarse<float>(*x, s, x->cs_variant)) != TH_OK) return st;
      // the tensor-core separator and spike products for 8 or more right-hand sides where built
      if (x->Sb16) x->cs_multi = 2;
      if ((st = tune_coarse_refine(*x, s)) != TH_OK) return st;
    } else if ((st = tune_coarse<double>(*x, s, x->cs_variant)) != TH_OK) {
      return st;
    }
  }
  TH_CU(cudaStreamSynchronize(s));
  {
    int flag = 0;
    TH_CU(cudaMemcpy(&flag, x->derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return TH_ERR_TIMEOUT;
  }
  TH_CU(cudaStreamSynchronize(s));
  *out = x.release();
  return TH_OK;
}

th_status th_set_kernel_variant(th_ctx* x, int kernel, int prec, int variant) {
  const int vmax = kernel == TH_K_DD ? (prec == TH_PREC_FP32 ? 5 : 3)
                   : kernel == TH_K_COARSE_REFINE ? 3
                   : (kernel == TH_K_COARSE_SOLVE || kernel == TH_K_CYCLE || kernel == TH_K_COARSE_MULTI) ? 2 : 1;
  if (!x || variant < 0 || variant > vmax || (prec != TH_PREC_FP64 && prec != TH_PREC_FP32))
    return TH_ERR_ARG;
  const bool d = (prec == TH_PREC_FP64);
  if (kernel == TH_K_FINE) {  // every right-hand-side count; FP32 also sets the double-single apply's
    if (d) {
      x->tc64 = x->tc64m = variant;
    } else {
      x->tc32 = x->tc32m = variant;
      x->tcds = x->tcdsm = variant;
    }
  } else if (kernel == TH_K_DD) {
    (d ? x->dds64 : x->dds32) = variant;
  } else if (kernel == TH_K_DD_BATCH) {
    x->dd_tc = variant;
  } else if (kernel == TH_K_COARSE_SOLVE) {
    x->cs_variant = variant;
  } else if (kernel == TH_K_RESID) {
    x->resid_ds = variant;
  } else if (kernel == TH_K_CYCLE) {
    x->fuse = variant;
  } else if (kernel == TH_K_COARSE_MULTI) {
    x->cs_multi = variant;
  } else if (kernel == TH_K_AZ) {
    x->az_ds = variant;
  } else if (kernel == TH_K_COARSE_REFINE) {
    x->coarse_refine = variant;
  } else if (kernel == TH_K_KRYLOV) {
    x->krylov_ds = variant;
  } else if (kernel == TH_K_SEP_SYM) {
    x->sep_sym = variant;
  } else {
    return TH_ERR_ARG;
  }
  ++x->epoch;
  return TH_OK;
}

th_status th_get_kernel_variant(const th_ctx* x, int kernel, int prec, int* variant) {
  if (!x || !variant || (prec != TH_PREC_FP64 && prec != TH_PREC_FP32)) return TH_ERR_ARG;
  const bool d = (prec == TH_PREC_FP64);
  if (kernel == TH_K_FINE) *variant = d ? x->tc64 : x->tc32;
  else if (kernel == TH_K_DD) *variant = d ? x->dds64 : x->dds32;
  else if (kernel == TH_K_DD_BATCH) *variant = (x->Wu && x->dd_tc) ? 1 : 0;
  else if (kernel == TH_K_COARSE_SOLVE) *variant = x->cs_variant;
  else if (kernel == TH_K_RESID) *variant = (x->resid_ds && x->kcds) ? 1 : 0;
  else if (kernel == TH_K_CYCLE) *variant = x->fuse;
  else if (kernel == TH_K_COARSE_MULTI) *variant = x->cs_multi;
  else if (kernel == TH_K_AZ) *variant = (x->az_ds && x->kcds && x->g.dim == 2) ? 1 : 0;
  else if (kernel == TH_K_COARSE_REFINE) *variant = (x->zc32 && x->wc32) ? x->coarse_refine : 0;
  else if (kernel == TH_K_KRYLOV) *variant = x->krylov_ds;
  else if (kernel == TH_K_SEP_SYM) *variant = (x->sep_sym && x->Ssym32) ? 1 : 0;
  else return TH_ERR_ARG;
  return TH_OK;
}

th_status th_device_status(th_ctx* x, void* stream) {
  if (!x) return TH_ERR_ARG;
  cudaStream_t s = S(stream);
  int flag = 0;
  TH_CU(cudaMemcpyAsync(&flag, x->derr, sizeof(int), cudaMemcpyDeviceToHost, s));
  TH_CU(cudaStreamSynchronize(s));
  if (!flag) return TH_OK;
  TH_CU(cudaMemsetAsync(x->derr, 0, sizeof(int), s));
  TH_CU(cudaStreamSynchronize(s));
  return TH_ERR_TIMEOUT;
}

th_status th_set_wait_limit(th_ctx* x, long long polls, void* stream) {
  if (!x) return TH_ERR_ARG;
  // status word 63 (see ptx.cuh): 0 = each kernel's default, > 0 = polls, < 0 = none
  const int word = polls < 0 ? 0 : (polls == 0 ? -1 : (int)std::min<long long>(polls, 1LL << 30));
  cudaStream_t s = S(stream);
  TH_CU(cudaMemcpyAsync(x->derr + 63, &word, sizeof(int), cudaMemcpyHostToDevice, s));
  TH_CU(cudaStreamSynchronize(s));
  return TH_OK;
}

th_status th_set_precision(th_ctx* x, int prec) {
  if (!x || prec < 0 || prec > 3) return TH_ERR_ARG;
  if (!has_prec(x->avail, prec)) return TH_ERR_UNSUPPORTED;
  x->active = prec;
  ++x->epoch;
  return TH_OK;
}

void th_destroy(th_ctx* x) { delete x; }

th_status th_launch_count(const th_ctx* x, long long* n) {
  if (!x || !n) return TH_ERR_ARG;
  *n = x->launches;
  return TH_OK;
}

th_status th_profile(th_ctx* x, int enable) {
  if (!x) return TH_ERR_ARG;
  if (enable) {
    x->prof_rec.clear();
    x->ev_used = 0;
  }
  x->prof_on = enable != 0;
  return TH_OK;
}

th_status th_profile_read(th_ctx* x, int kind, double* ms, long long* launches) {
  if (!x || !ms || !launches || kind < 0 || kind >= TH_K_COUNT) return TH_ERR_ARG;
  double tot = 0.0;
  long long cnt = 0;
  for (const auto& r : x->prof_rec) {
    if (r.first != kind) continue;
    TH_CU(cudaEventSynchronize(x->ev_pool[r.second + 1]));
    float t = 0.0f;
    TH_CU(cudaEventElapsedTime(&t, x->ev_pool[r.second], x->ev_pool[r.second + 1]));
    tot += t;
    ++cnt;
  }
  *ms = tot;
  *launches = cnt;
  return TH_OK;
}

th_status th_apply(th_ctx* x, int op, const double* xin, double* y, int nrhs, int prec, void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!xin || !y || (prec != TH_PREC_FP64 && prec != TH_PREC_FP32)) return TH_ERR_ARG;
  cudaStream_t s = S(stream);
  const double2* in = reinterpret_cast<const double2*>(xin);
  double2* out = reinterpret_cast<double2*>(y);
  if (op == TH_OP_A || op == TH_OP_AS) {
    if (prec == TH_PREC_FP64) return fine_apply<double>(*x, op, in, nullptr, out, nrhs, s);
    if (!x->mixed) return TH_ERR_UNSUPPORTED;
    const long long n = x->g.N * (long long)nrhs;
    if ((st = narrow(*x, in, x->f32, n, s)) != TH_OK) return st;
    if ((st = fine_apply<float>(*x, op, x->f32, nullptr, x->r32, nrhs, s)) != TH_OK) return st;
    return widen(*x, x->r32, out, n, 0, s);
  }
  if (op == TH_OP_AQ) {
    if (prec == TH_PREC_FP64) return coarse_apply_<double>(*x, in, out, nrhs, s);
    if (!x->mixed) return TH_ERR_UNSUPPORTED;
    const long long n = x->g.Nc * (long long)nrhs;
    if ((st = narrow(*x, in, x->rc32, n, s)) != TH_OK) return st;
    if ((st = coarse_apply_<float>(*x, x->rc32, x->uc32, nrhs, s)) != TH_OK) return st;
    return widen(*x, x->uc32, out, n, 0, s);
  }
  return TH_ERR_ARG;
}

th_status th_residual(th_ctx* x, const double* f, const double* u, double* r, int nrhs, void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!f || !u || !r) return TH_ERR_ARG;
  return fine_apply<double>(*x, TH_OP_A, reinterpret_cast<const double2*>(u), reinterpret_cast<const double2*>(f),
                            reinterpret_cast<double2*>(r), nrhs, S(stream));
}

th_status th_residual_mixed(th_ctx* x, const double* f, const double* u, float* r, int nrhs, void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!f || !u || !r) return TH_ERR_ARG;
  if (!x->mixed) return TH_ERR_UNSUPPORTED;
  return outer_residual(*x, reinterpret_cast<const double2*>(u), reinterpret_cast<const double2*>(f),
                        reinterpret_cast<float2*>(r), nrhs, S(stream));
}

th_status th_smooth(th_ctx* x, const double* f, double* u, int nrhs, void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!f || !u) return TH_ERR_ARG;
  cudaStream_t s = S(stream);
  const double2* f2 = reinterpret_cast<const double2*>(f);
  double2* u2 = reinterpret_cast<double2*>(u);
  if (x->active == TH_PREC_FP64) return smooth<double>(*x, TH_PREC_FP64, f2, u2, false, nrhs, s);
  // mixed: u += S(0, f - A u) in FP32
  const long long n = x->g.N * (long long)nrhs;
  if ((st = outer_residual(*x, u2, f2, x->f32, nrhs, s)) != TH_OK) return st;
  if ((st = smooth<float>(*x, x->active, x->f32, x->u32, true, nrhs, s)) != TH_OK) return st;
  return widen(*x, x->u32, u2, n, 1, s);
}

th_status th_restrict(th_ctx* x, const double* r, double* rc, int nrhs, void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!r || !rc) return TH_ERR_ARG;
  return restrict_<double>(*x, reinterpret_cast<const double2*>(r), reinterpret_cast<double2*>(rc), nrhs, S(stream));
}

th_status th_prolong(th_ctx* x, const double* uc, double* u, double omega, int nrhs, void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!uc || !u) return TH_ERR_ARG;
  return prolong_<double>(*x, reinterpret_cast<const double2*>(uc), reinterpret_cast<double2*>(u), omega, nrhs,
                          S(stream));
}

th_status th_coarse_solve(th_ctx* x, const double* rc, double* uc, int nrhs, void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!rc || !uc) return TH_ERR_ARG;
  cudaStream_t s = S(stream);
  const double2* in = reinterpret_cast<const double2*>(rc);
  double2* out = reinterpret_cast<double2*>(uc);
  if (x->active == TH_PREC_FP64) return coarse_solve_<double>(*x, in, out, nrhs, s);
  const long long n = x->g.Nc * (long long)nrhs;
  if ((st = narrow(*x, in, x->rc32, n, s)) != TH_OK) return st;
  if ((st = coarse_solve_<float>(*x, x->rc32, x->uc32, nrhs, s)) != TH_OK) return st;
  return widen(*x, x->uc32, out, n, 0, s);
}

th_status th_cycle(th_ctx* x, const double* f, double* u, int nrhs, void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!f || !u) return TH_ERR_ARG;
  cudaStream_t s = S(stream);
  const double2* f2 = reinterpret_cast<const double2*>(f);
  double2* u2 = reinterpret_cast<double2*>(u);
  if (x->active == TH_PREC_FP64) return cycle<double>(*x, TH_PREC_FP64, f2, u2, false, nrhs, s);
  // mixed: TwoGridStep(u, f) = u + TwoGridStep(0, f - A u) (the step is affine in u and f)
  const long long n = x->g.N * (long long)nrhs;
  if ((st = outer_residual(*x, u2, f2, x->f32, nrhs, s)) != TH_OK) return st;
  if (can_fuse<float>(*x, true)) return cycle_fused<float>(*x, x->active, x->f32, x->u32, nrhs, u2, 1, s);
  if ((st = cycle<float>(*x, x->active, x->f32, x->u32, true, nrhs, s)) != TH_OK) return st;
  return widen(*x, x->u32, u2, n, 1, s);
}

th_status th_cycle_graph(th_ctx* x, const double* f, double* u, int nrhs, void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!f || !u) return TH_ERR_ARG;
  if (!x->use_graphs || x->prof_on) return th_cycle(x, f, u, nrhs, stream);
  return graph_run(*x, 0, f, u, nrhs, S(stream),
                   [&](cudaStream_t gs) { return th_cycle(x, f, u, nrhs, (void*)gs); });
}

th_status th_set_graphs(th_ctx* x, int enable) {
  if (!x || (enable != 0 && enable != 1)) return TH_ERR_ARG;
  x->use_graphs = enable != 0;
  if (!enable) x->drop_graphs();
  return TH_OK;
}

// ------------------------------------------------------------ learned coarse corrector
th_status th_unet_param_count(int levels, int base, size_t* n) {
  if (!n || !th::UNet::check(levels, base)) return TH_ERR_ARG;
  *n = th::UNet::param_count(levels, base);
  return TH_OK;
}

th_status th_unet_init(th_ctx* x, int levels, int base, int batch_max, const float* params, size_t n,
                       void* stream) {
  if (!x || !params || batch_max < 1 || !th::UNet::check(levels, base)) return TH_ERR_ARG;
  if (n != th::UNet::param_count(levels, base)) return TH_ERR_ARG;
  if (x->mesh.dim != 2 || x->gal) return TH_ERR_UNSUPPORTED;  // trained on the QSFEM coarse operator
  const th::Geometry& g = x->g;
  // eta = k h_c at the coarse nodes: mean over the adjacent coarse cells, each
  // of which takes the k of the fine cell containing it
  const int nc = g.nc, m = g.mc;
  std::vector<float> eta((size_t)m * m);
  for (int y = 0; y < m; ++y)
    for (int xx = 0; xx < m; ++xx) {
      double acc = 0;
      int cnt = 0;
      for (int cy = y - 1; cy <= y; ++cy)
        for (int cx = xx - 1; cx <= xx; ++cx) {
          if (cy < 0 || cy >= nc || cx < 0 || cx >= nc) continue;
          acc += x->k_host[(size_t)(cy / g.q) * g.n + cx / g.q] * g.hc;
          ++cnt;
        }
      eta[(size_t)y * m + xx] = (float)(acc / cnt);
    }
  delete x->unet;
  x->unet = new (std::nothrow) th::UNet(levels, base, batch_max, m, eta, x->derr);
  if (!x->unet || !x->unet->ok()) {
    delete x->unet;
    x->unet = nullptr;
    return TH_ERR_NOMEM;
  }
  if (x->unet->set_params(params, S(stream)) != cudaSuccess) return TH_ERR_CUDA;
  ++x->epoch;
  return TH_OK;
}

th_status th_unet_get_params(th_ctx* x, float* params, size_t n, void* stream) {
  if (!x || !params) return TH_ERR_ARG;
  if (!x->unet) return TH_ERR_UNSUPPORTED;
  if (n != x->unet->nparams()) return TH_ERR_ARG;
  return cuda_status(x->unet->get_params(params, S(stream)));
}

th_status th_unet_set_params(th_ctx* x, const float* params, size_t n, void* stream) {
  if (!x || !params) return TH_ERR_ARG;
  if (!x->unet) return TH_ERR_UNSUPPORTED;
  if (n != x->unet->nparams()) return TH_ERR_ARG;
  return cuda_status(x->unet->set_params(params, S(stream)));
}

th_status th_unet_forward(th_ctx* x, const float* in_dev, float* out_dev, int batch, void* stream) {
  if (!x || !in_dev || !out_dev) return TH_ERR_ARG;
  if (!x->unet) return TH_ERR_UNSUPPORTED;
  if (batch < 1 || batch > x->unet->batch_max()) return TH_ERR_ARG;
  return cuda_status(x->unet->forward_from(in_dev, out_dev, batch, S(stream)));
}

th_status th_unet_backward(th_ctx* x, const float* gout_dev, float* grads_dev, int batch, void* stream) {
  if (!x || !gout_dev || !grads_dev) return TH_ERR_ARG;
  if (!x->unet) return TH_ERR_UNSUPPORTED;
  if (batch < 1 || batch > x->unet->batch_max()) return TH_ERR_ARG;
  return cuda_status(x->unet->backward_to(gout_dev, grads_dev, batch, S(stream)));
}

th_status th_unet_train_step(th_ctx* x, const double* rc_dev, const double* uc_dev, int batch, double lr,
                             double* loss, void* stream) {
  if (!x || !rc_dev || !uc_dev || !(lr > 0)) return TH_ERR_ARG;
  if (!x->unet) return TH_ERR_UNSUPPORTED;
  if (batch < 1 || batch > x->unet->batch_max()) return TH_ERR_ARG;
  return cuda_status(x->unet->train_step(reinterpret_cast<const double2*>(rc_dev),
                                         reinterpret_cast<const double2*>(uc_dev), batch, lr, loss, S(stream)));
}

th_status th_unet_correct(th_ctx* x, const double* rc_dev, double* uc_dev, int nrhs, void* stream) {
  if (!x || !rc_dev || !uc_dev || nrhs < 1) return TH_ERR_ARG;
  if (!x->unet) return TH_ERR_UNSUPPORTED;
  x->launches += x->unet->launches_per_forward() * ((nrhs + x->unet->batch_max() - 1) / x->unet->batch_max());
  return cuda_status(x->unet->correct<double2>(reinterpret_cast<const double2*>(rc_dev),
                                               reinterpret_cast<double2*>(uc_dev), x->g.Nc, nrhs, S(stream)));
}

th_status th_set_coarse(th_ctx* x, int mode, int plain_iters) {
  if (!x || mode < 0 || mode > 2 || plain_iters < 0) return TH_ERR_ARG;
  if (mode == 1 && !x->unet) return TH_ERR_UNSUPPORTED;
  x->coarse_mode = mode;
  x->plain_iters = plain_iters;
  ++x->epoch;
  return TH_OK;
}

th_status th_cycle_host(th_ctx* x, const double* f_host, double* u_host, int nrhs, void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!f_host || !u_host) return TH_ERR_ARG;
  cudaStream_t s = S(stream);
  const size_t nb = sizeof(double2) * x->g.N * (size_t)nrhs;
  TH_CU(cudaMemcpyAsync(x->fin, f_host, nb, cudaMemcpyHostToDevice, s));
  TH_CU(cudaMemcpyAsync(x->uin, u_host, nb, cudaMemcpyHostToDevice, s));
  if ((st = th_cycle_graph(x, (const double*)x->fin, (double*)x->uin, nrhs, stream)) != TH_OK) return st;
  TH_CU(cudaMemcpyAsync(u_host, x->uin, nb, cudaMemcpyDeviceToHost, s));
  TH_CU(cudaStreamSynchronize(s));
  return TH_OK;
}

th_status th_solve(th_ctx* x, const double* f, double* u, int nrhs, th_solve_info* info, void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!f || !u) return TH_ERR_ARG;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = S(stream);
  const th::Geometry& g = x->g;
  const long long N = g.N;
  const int m = x->prm.restart;
  if (!x->pin && cudaHostAlloc(&x->pin, sizeof(double) * 2 * 5 * x->prm.nrhs_max, cudaHostAllocDefault) != cudaSuccess)
    return TH_ERR_NOMEM;
  const long long vstride = N * (long long)nrhs;  // between basis vectors
  const double2* f2 = reinterpret_cast<const double2*>(f);
  double2* u2 = reinterpret_cast<double2*>(u);
  const double tol = x->prm.tol;
  // the mixed forms' Gram-Schmidt products in double-single arithmetic (the FP64 form stays FP64)
  const bool kds = x->krylov_ds && x->active != TH_PREC_FP64;
  std::vector<double> fn, beta;
  if ((st = norms(*x, f2, nrhs, fn, s)) != TH_OK) return st;
  for (double v : fn)
    if (!std::isfinite(v)) return TH_ERR_NONFINITE;
  std::vector<int> done(nrhs, 0), its(nrhs, 0);
  for (int r = 0; r < nrhs; ++r)
    if (fn[r] == 0.0) done[r] = 1;
  std::vector<cplx> H((size_t)nrhs * (m + 1) * m), cs((size_t)nrhs * m), sn((size_t)nrhs * m),
      gg((size_t)nrhs * (m + 1));
  std::vector<double> scal(nrhs);
  std::vector<double2> yv;
  int it = 0;
  th_status result = TH_OK;
  // learned corrector: fall back to the direct coarse solve once the iteration
  // count reaches 1.5 x the plain count (restart from the current iterate)
  const int saved_mode = x->coarse_mode;
  const int limit = (saved_mode == 1 && x->plain_iters > 0) ? (int)std::ceil(1.5 * x->plain_iters) : INT32_MAX;
  int fallbacks = 0;
  bool switch_now = false;
  struct Restore {
    th_ctx* x;
    int mode;
    ~Restore() {
      if (x->coarse_mode != mode) {
        x->coarse_mode = mode;
        ++x->epoch;
      }
    }
  } restore{x, saved_mode};
  // the residual at the loop's exit, FP64 (reused as the final true residual)
  bool exact_exit = false;
  for (;;) {
    // r = f - A x -> V_0: in double-single arithmetic in the mixed forms (about
    // 2^-44 of |A||x|); when that shows convergence or the iteration limit, again
    // in FP64, which decides
    const std::vector<int> done_before = done;
    bool all = true;
    for (int pass = 0; pass < 2; ++pass) {
      const bool exact = pass == 1 || !kds;
      if ((st = fgmres_residual(*x, u2, f2, x->Vk, nrhs, s, exact)) != TH_OK) return st;
      if ((st = norms(*x, x->Vk, nrhs, beta, s)) != TH_OK) return st;
      done = done_before;
      all = true;
      for (int r = 0; r < nrhs; ++r) {
        if (!std::isfinite(beta[r])) return TH_ERR_NONFINITE;
        if (!done[r] && beta[r] <= tol * fn[r]) done[r] = 1;
        all = all && done[r];
      }
      exact_exit = exact;
      if (exact || !(all || it >= x->prm.maxit)) break;
    }
    if (all || it >= x->prm.maxit) break;
    std::vector<int> active(nrhs), jr(nrhs, 0);
    for (int r = 0; r < nrhs; ++r) {
      active[r] = !done[r];
      scal[r] = active[r] ? 1.0 / beta[r] : 0.0;
      std::fill(gg.begin() + (size_t)r * (m + 1), gg.begin() + (size_t)(r + 1) * (m + 1), cplx(0.0));
      gg[(size_t)r * (m + 1)] = beta[r];
    }
    // device Arnoldi state for this restart cycle
    {
      std::vector<double2> g0((size_t)nrhs * (m + 1), make_double2(0.0, 0.0));
      for (int r = 0; r < nrhs; ++r) g0[(size_t)r * (m + 1)] = make_double2(beta[r], 0.0);
      TH_CU(cudaMemcpyAsync(x->gd, g0.data(), sizeof(double2) * g0.size(), cudaMemcpyHostToDevice, s));
      TH_CU(cudaMemcpyAsync(x->actd, active.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
      TH_CU(cudaMemcpyAsync(x->fnd, fn.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
      TH_CU(cudaMemcpyAsync(x->scal, scal.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
      // the host buffers are read by the copies above: finish them before they change
      TH_CU(cudaStreamSynchronize(s));
    }
    x->launches += 1;
    // the basis in the split form of the double-single Gram-Schmidt kernels (mixed forms)
    if (kds) {
      TH_CU(th::launch_scale_split(x->Vk, x->Vk, x->scal, N, nrhs, s));
    } else {
      TH_CU(th::launch_scale_rhs(x->Vk, x->Vk, x->scal, N, nrhs, s));
    }
    th::ArnoldiArgs aa{x->h1, x->nrm, x->Hd, x->csd, x->snd, x->gd, x->fnd, x->actd, x->scal, x->statd, tol, nrhs, m};
    // Arnoldi steps are enqueued one ahead of the host: after enqueueing step j the
    // host reads the status of step j - 1 (pinned copy, event), so the GPU does not
    // wait for the host between steps.  When the residual estimates predict that
    // step j converges, the host reads its status before enqueueing step j + 1, so
    // that no step is enqueued after the last one in the usual case.
    cudaEvent_t evs[2];
    TH_CU(cudaEventCreateWithFlags(&evs[0], cudaEventDisableTiming));
    if (cudaEventCreateWithFlags(&evs[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaEventDestroy(evs[0]);
      return TH_ERR_CUDA;
    }
    struct EvGuard {
      cudaEvent_t* e;
      ~EvGuard() {
        cudaEventDestroy(e[0]);
        cudaEventDestroy(e[1]);
      }
    } evguard{evs};
    const int room = std::max(0, std::min(m, x->prm.maxit - it));
    int jdone = 0, it_cycle = 0, last_read = -1;
    bool stop = false, expect_conv = false;
    std::vector<double> stj((size_t)nrhs * 5), rel_prev(nrhs, -1.0), rel_last(nrhs, -1.0);
    auto read_status = [&](int jj) -> th_status {
      TH_CU(cudaEventSynchronize(evs[jj & 1]));
      std::memcpy(stj.data(), x->pin + (size_t)(jj & 1) * nrhs * 5, sizeof(double) * nrhs * 5);
      last_read = jj;
      bool any = false, cancel = false;
      for (int r = 0; r < nrhs; ++r) {
        const double* sr = &stj[(size_t)r * 5];
        if (sr[3] != 0.0) return TH_ERR_NONFINITE;
        if (active[r]) {
          jr[r] = (int)sr[1];
          its[r] = it + jj + 1;
          if (sr[2] != 0.0) cancel = true;
          if (sr[0] == 0.0) active[r] = 0;
          rel_prev[r] = rel_last[r];
          rel_last[r] = sr[4];
        }
        any = any || active[r];
      }
      jdone = jj + 1;
      it_cycle = jj + 1;
      if (!any || cancel || it + jj + 1 >= x->prm.maxit) stop = true;
      if (x->coarse_mode == 1 && it + jj + 1 >= limit) {
        switch_now = true;
        stop = true;
      }
      // does the next step reach the tolerance for every active rhs (geometric extrapolation)?
      expect_conv = any;
      for (int r = 0; r < nrhs; ++r) {
        if (!active[r]) continue;
        const double q = (rel_prev[r] > 0.0 && rel_last[r] > 0.0) ? std::min(1.0, rel_last[r] / rel_prev[r]) : 1.0;
        if (!(rel_last[r] * q <= 3.0 * tol)) expect_conv = false;
      }
      return TH_OK;
    };
    for (int j = 0; j < room && !stop; ++j) {
      if (expect_conv && last_read < j - 1) {  // the step before this one may have converged
        if ((st = read_status(j - 1)) != TH_OK) return st;
        if (stop) break;
      }
      double2* Vj = x->Vk + (size_t)j * vstride;
      double2* Zj = x->Zk + (size_t)j * vstride;
      // one Arnoldi step: z_j = B v_j, w = A z_j, one classical Gram-Schmidt pass
      // (the coefficients and ||w||^2 before it), then ||w||^2 after it, the
      // Hessenberg column and rotations, v_{j+1}, and the step's status copied to
      // pinned host memory.  A pass that cancels more than 99.99 % of ||w||^2 makes
      // the host restart (loss of orthogonality ~ eps ||w||^2 / ||w - V h||^2),
      // which with the two-grid preconditioner does not occur in practice.
      // blocks per right-hand side of the double-single dots and norms: with
      // many right-hand sides a quarter as many, so each thread sums about four
      // times the entries before the block reduction (its fixed cost)
      const int nbk = nrhs >= 8 ? std::max(1, x->nblk / 4) : x->nblk;
      auto step = [&](cudaStream_t ss) -> th_status {
        th_status e;
        if ((e = precondition(*x, Vj, Zj, nrhs, ss, kds)) != TH_OK) return e;
        if ((e = az_apply(*x, Zj, x->w, nrhs, ss)) != TH_OK) return e;
        x->launches += 6;
        {
          Prof prof(*x, TH_K_KRYLOV, ss);
          if (kds) {
            TH_CU(th::launch_mdot_ds(x->Vk, vstride, x->w, N, j + 1, 1, nrhs, x->dpart, x->h1, nbk, 1, ss));
            TH_CU(th::launch_maxpy_ds(x->Vk, vstride, x->h1, j + 2, x->w, N, j + 1, nrhs, -1.0, 1, ss));
            TH_CU(th::launch_norm2_ds(x->w, N, nrhs, x->npart, x->nrm, nbk, ss));
          } else {
            TH_CU(th::launch_mdot(x->Vk, vstride, x->w, N, j + 1, 1, nrhs, x->dpart, x->h1, x->nblk, ss));
            TH_CU(th::launch_maxpy(x->Vk, vstride, x->h1, j + 2, x->w, N, j + 1, nrhs, -1.0, ss));
            TH_CU(th::launch_norm2(x->w, N, nrhs, x->npart, x->nrm, x->nblk, ss));
          }
          TH_CU(th::launch_arnoldi(aa, j, ss));
          if (kds) {
            TH_CU(th::launch_scale_split(x->w, x->Vk + (size_t)(j + 1) * vstride, x->scal, N, nrhs, ss));
          } else {
            TH_CU(th::launch_scale_rhs(x->w, x->Vk + (size_t)(j + 1) * vstride, x->scal, N, nrhs, ss));
          }
        }
        TH_CU(cudaMemcpyAsync(x->pin + (size_t)(j & 1) * nrhs * 5, x->statd, sizeof(double) * nrhs * 5,
                              cudaMemcpyDeviceToHost, ss));
        return TH_OK;
      };
      // the whole step from one CUDA graph per (j, buffers): a launch instead of a
      // dozen, and no launch gaps between its small Krylov kernels
      st = (x->use_graphs && !x->prof_on) ? graph_run(*x, 3 + 2 * j, Vj, Zj, nrhs, s, step) : step(s);
      if (st != TH_OK) return st;
      TH_CU(cudaEventRecord(evs[j & 1], s));
      if (j >= 1 && last_read < j - 1 && (st = read_status(j - 1)) != TH_OK) return st;
    }
    if (!stop && room > 0 && last_read < room - 1 && (st = read_status(room - 1)) != TH_OK) return st;
    it += it_cycle;
    // the Hessenberg columns and g of the valid steps (a discarded step touches neither)
    const int jmax = jdone;
    std::vector<double2> Hh((size_t)nrhs * (m + 1) * m), gh((size_t)nrhs * (m + 1));
    if (jmax > 0) {
      TH_CU(cudaMemcpyAsync(Hh.data(), x->Hd, sizeof(double2) * Hh.size(), cudaMemcpyDeviceToHost, s));
      TH_CU(cudaMemcpyAsync(gh.data(), x->gd, sizeof(double2) * gh.size(), cudaMemcpyDeviceToHost, s));
      TH_CU(cudaStreamSynchronize(s));
    }
    for (size_t q = 0; q < H.size(); ++q) H[q] = cplx(Hh[q].x, Hh[q].y);
    for (size_t q = 0; q < gg.size(); ++q) gg[q] = cplx(gh[q].x, gh[q].y);
    for (int r = 0; r < nrhs; ++r) jr[r] = std::min(jr[r], jmax);
    const int jdone_all = jmax;
    // x += Z y per right-hand side (y = 0 beyond its own last step)
    jdone = jdone_all;
    yv.assign((size_t)nrhs * jdone, make_double2(0, 0));
    for (int r = 0; r < nrhs; ++r) {
      const int jj = jr[r];
      if (jj == 0) continue;
      const cplx* Hc = &H[((size_t)r * (m + 1)) * m];
      const cplx* gr = &gg[(size_t)r * (m + 1)];
      std::vector<cplx> y(jj);
      for (int i = jj - 1; i >= 0; --i) {
        cplx sacc = gr[i];
        for (int k = i + 1; k < jj; ++k) sacc -= Hc[i + (size_t)k * (m + 1)] * y[k];
        const cplx d = Hc[i + (size_t)i * (m + 1)];
        if (d == 0.0) return TH_ERR_BREAKDOWN;
        y[i] = sacc / d;
      }
      for (int i = 0; i < jj; ++i) yv[(size_t)r * jdone + i] = make_double2(y[i].real(), y[i].imag());
    }
    TH_CU(cudaMemcpyAsync(x->ybuf, yv.data(), sizeof(double2) * yv.size(), cudaMemcpyHostToDevice, s));
    x->launches += 1;
    if (kds) {
      TH_CU(th::launch_maxpy_ds(x->Zk, vstride, x->ybuf, jdone, u2, N, jdone, nrhs, 1.0, 0, s));
    } else {
      TH_CU(th::launch_maxpy(x->Zk, vstride, x->ybuf, jdone, u2, N, jdone, nrhs, 1.0, s));
    }
    TH_CU(cudaStreamSynchronize(s));
    if (switch_now) {
      switch_now = false;
      x->coarse_mode = 0;
      ++x->epoch;
      ++fallbacks;
    }
  }
  // final true residuals (FP64): those of the loop's exit
  std::vector<double> rn = beta;
  if (!exact_exit) {
    if ((st = fine_apply<double>(*x, TH_OP_A, u2, f2, x->w, nrhs, s)) != TH_OK) return st;
    if ((st = norms(*x, x->w, nrhs, rn, s)) != TH_OK) return st;
  }
  double rmax = 0.0;
  int nconv = 0;
  for (int r = 0; r < nrhs; ++r) {
    const double rel = fn[r] > 0 ? rn[r] / fn[r] : 0.0;
    rmax = std::max(rmax, rel);
    if (rel <= tol * 1.0000001 || fn[r] == 0.0) ++nconv;
  }
  if (nconv < nrhs) result = TH_ERR_NOCONV;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = it;
    info->converged = nconv;
    info->relres_max = rmax;
    for (int r = 0; r < nrhs && r < 64; ++r) info->iters_per_rhs[r] = its[r];
    info->fallbacks = fallbacks;
    info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return result;
}

th_status th_solve_host(th_ctx* x, const double* f_host, double* u_host, int nrhs, th_solve_info* info,
                        void* stream) {
  th_status st = check_nrhs(x, nrhs);
  if (st != TH_OK) return st;
  if (!f_host || !u_host) return TH_ERR_ARG;
  cudaStream_t s = S(stream);
  const size_t nb = sizeof(double2) * x->g.N * (size_t)nrhs;
  TH_CU(cudaMemcpyAsync(x->fin, f_host, nb, cudaMemcpyHostToDevice, s));
  TH_CU(cudaMemcpyAsync(x->uin, u_host, nb, cudaMemcpyHostToDevice, s));
  th_status rs = th_solve(x, (const double*)x->fin, (double*)x->uin, nrhs, info, stream);
  if (rs != TH_OK && rs != TH_ERR_NOCONV) return rs;
  TH_CU(cudaMemcpyAsync(u_host, x->uin, nb, cudaMemcpyDeviceToHost, s));
  TH_CU(cudaStreamSynchronize(s));
  return rs;
}

// ------------------------------------------------------------ host-only
th_status th_host_reference_1d(int p, double* nodes, double* mass, double* stiff) {
  if (p < 1 || p > th::kMaxP || !nodes || !mass || !stiff) return TH_ERR_ARG;
  if (p % 2 != 0) return TH_ERR_ARG;
  th::Ref1D r = th::reference_1d(p);
  std::copy(r.nodes.begin(), r.nodes.end(), nodes);
  std::copy(r.M.begin(), r.M.end(), mass);
  std::copy(r.K.begin(), r.K.end(), stiff);
  return TH_OK;
}

th_status th_host_qsfem_cell(double k, double eps, double hc, double* out) {
  if (!out || !(k > 0) || !(hc > 0)) return TH_ERR_ARG;
  cplx d[3];
  th::qsfem_cell(k, eps, hc, d);
  for (int i = 0; i < 3; ++i) {
    out[2 * i] = d[i].real();
    out[2 * i + 1] = d[i].imag();
  }
  return TH_OK;
}

th_status th_host_qsfem27_cell(double k, double eps, double hc, double* out) {
  if (!out || !(hc > 0) || !(k > 0) || !(eps >= 0)) return TH_ERR_ARG;
  cplx d[4];
  th::qsfem27_cell(k, eps, hc, d);
  for (int i = 0; i < 4; ++i) {
    out[2 * i] = d[i].real();
    out[2 * i + 1] = d[i].imag();
  }
  return TH_OK;
}

th_status th_host_inverse_rows(const th_mesh* mesh, const double* k_host, const double* eps_host,
                               const th_params* prm, int sub, int* box, double* out, size_t out_len) {
  if (!mesh || !prm || !k_host || !box || !out) return TH_ERR_ARG;
  th::Geometry g;
  th_status st = th::make_geometry(*mesh, *prm, g);
  if (st != TH_OK) return st;
  if (sub < 0 || sub >= g.nsub) return TH_ERR_ARG;
  if (out_len < (size_t)g.NR * g.NC * 2) return TH_ERR_NOMEM;
  std::copy(&g.box[(size_t)sub * th::kBox], &g.box[(size_t)sub * th::kBox] + th::kBox, box);
  th::Ref1D ref = th::reference_1d(mesh->p);
  std::vector<cplx> o((size_t)g.NR * g.NC);
  if ((st = th::subdomain_inverse_rows(g, ref, k_host, eps_host, prm->alpha_s, sub, o.data())) != TH_OK) return st;
  std::memcpy(out, o.data(), o.size() * sizeof(cplx));
  return TH_OK;
}

}  // extern "C"

th_status th_host_coarse_separators(const th_mesh* mesh, const double* k_host, const double* eps_host,
                                    const th_params* prm, int P, int* sep, double* sinv, size_t sinv_len) {
  if (!mesh || !prm || !k_host || !sep || !sinv) return TH_ERR_ARG;
  if (mesh->dim != 2) return TH_ERR_UNSUPPORTED;
  th::Geometry g;
  th_status st = th::make_geometry(*mesh, *prm, g);
  if (st != TH_OK) return st;
  if (P < 2 || 2 * P - 1 > g.mc) return TH_ERR_ARG;
  const size_t nred = (size_t)(P - 1) * g.mc;
  if (sinv_len < 2 * nred * nred) return TH_ERR_NOMEM;
  std::vector<double> zero;
  const double* eps = eps_host;
  if (!eps) {
    zero.assign((size_t)g.n * g.n, 0.0);
    eps = zero.data();
  }
  th::CoarseBlocks cb;
  if ((st = th::coarse_setup(g, k_host, eps, cb, false)) != TH_OK) return st;
  th::CoarsePart cp;
  if ((st = th::coarse_partition(g, cb, P, cp)) != TH_OK) return st;
  for (int k = 0; k < P - 1; ++k) sep[k] = cp.sep[k];
  std::memcpy(sinv, cp.Sinv.data(), nred * nred * sizeof(cplx));
  return TH_OK;
}

th_status th_host_galerkin(const th_mesh* mesh, const double* k_host, const double* eps_host,
                           const th_params* prm, double* stencil, size_t stencil_len, const double* b, double* xo) {
  if (!mesh || !prm || !k_host || !stencil) return TH_ERR_ARG;
  if (mesh->dim != 2) return TH_ERR_UNSUPPORTED;
  th::Geometry g;
  th_status st = th::make_geometry(*mesh, *prm, g);
  if (st != TH_OK) return st;
  const int q = g.q, mc = g.mc, S = 2 * q + 1;
  if (stencil_len < (size_t)2 * mc * mc * S * S) return TH_ERR_NOMEM;
  th::GalBlocks gb;
  if ((st = th::galerkin_setup(g, k_host, eps_host, prm->alpha_c, gb)) != TH_OK) return st;
  std::memcpy(stencil, gb.st.data(), gb.st.size() * sizeof(cplx));
  if (!b || !xo) return TH_OK;
  // the device sweep's arithmetic on the host: forward x_j = G_j (b_j - L_j x_{j-1}),
  // backward x_j -= G_j U_j x_{j+1}
  const size_t Nc = (size_t)mc * mc;
  std::vector<cplx> x(Nc, cplx(0.0)), t;
  const cplx* B = reinterpret_cast<const cplx*>(b);
  for (int dir = 0; dir < 2; ++dir)
    for (int jj = 0; jj < g.n - dir; ++jj) {
      const int j = dir ? g.n - 2 - jj : jj;
      const int lo = th::gal_row_lo(j, q), hi = th::gal_row_hi(j, q), Sj = (hi - lo + 1) * mc;
      int nlo = 0, nhi = -1;
      if (!dir && j > 0) { nlo = th::gal_row_lo(j - 1, q); nhi = lo - 1; }
      if (dir && j + 1 < g.n) { nlo = hi + 1; nhi = th::gal_row_hi(j + 1, q); }
      t.assign(Sj, cplx(0.0));
      for (int i = 0; i < Sj; ++i) {
        const int y = lo + i / mc, xx = i % mc;
        cplx acc = 0.0;
        for (int dy = std::max(-q, nlo - y); dy <= std::min(q, nhi - y); ++dy)
          for (int dx = std::max(-q, -xx); dx <= std::min(q, mc - 1 - xx); ++dx)
            acc += gb.st[((size_t)y * mc + xx) * S * S + (dy + q) * S + dx + q] * x[(size_t)(y + dy) * mc + xx + dx];
        t[i] = dir ? acc : B[(size_t)lo * mc + i] - acc;
      }
      const cplx* G = gb.G.data() + th::gal_goff(j, q, mc);
      for (int r = 0; r < Sj; ++r) {
        cplx v = 0.0;
        for (int c = 0; c < Sj; ++c) v += G[(size_t)r * Sj + c] * t[c];
        if (dir) x[(size_t)lo * mc + r] -= v;
        else x[(size_t)lo * mc + r] = v;
      }
    }
  std::memcpy(xo, x.data(), Nc * sizeof(cplx));
  return TH_OK;
}
