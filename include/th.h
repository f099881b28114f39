/*
 * th.h -- C ABI of the GB300 two-grid Helmholtz library.
 *
 * The method (Stolk, "A two-grid method with dispersion matching for
 * finite-element Helmholtz problems"): the Helmholtz equation
 *     -Lap u - (k^2 + i eps) u = f              (Section 2, Eq. Helmholtz_eq)
 * on the unit square with Robin (absorbing) or Neumann sides, discretised with
 * continuous Q_p elements on a uniform mesh of n x n cells (Section 3.1,
 * Eq. bilin_form), is solved by flexible GMRES preconditioned with the
 * two-grid step of Algorithm 1: a complex-shifted overlapping domain-
 * decomposition smoother (Algorithm 2, Eq. RAS_like_update) and a coarse
 * correction on a mesh of spacing 2h/p with the dispersion-minimising QSFEM
 * 9-point operator (Sections 3.2-3.3, Eq. P_QSFEM, Eq. element_wise_qsfem).
 *
 * Conventions shared by every entry point
 *   - Fine vectors hold N = (n p + 1)^2 complex values, lexicographic on the
 *     global node grid, x fastest; coarse vectors hold Nc = (n p / 2 + 1)^2.
 *     The nodal basis is the Lagrange basis on the Gauss-Lobatto-Legendre
 *     points of each cell.
 *   - Complex numbers are interleaved (re, im) IEEE doubles: a vector is a
 *     double[2 N].  Several right-hand sides are stored one after another:
 *     rhs r starts at element 2 N r.
 *   - Pointers named *_dev are CUDA device pointers (or managed memory);
 *     pointers named *_host are host pointers (pageable or pinned).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Calls are asynchronous with respect to the host unless stated.
 *   - The caller owns every buffer it passes.  The library never frees caller
 *     memory and allocates no device memory except inside th_setup's caller-
 *     provided workspace (plus what the CUDA runtime itself reserves).
 *   - Errors are reported by the return code only (no exceptions, no aborts).
 *     After an error the outputs are unspecified; the context stays valid for
 *     th_destroy.  th_status_str gives a static message.
 *   - One context must not be used from two host threads at once.
 */
#ifndef TH_H
#define TH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TH_OK = 0,
  TH_ERR_ARG = 1,          /* invalid argument or size */
  TH_ERR_CUDA = 2,         /* a CUDA runtime call or kernel launch failed */
  TH_ERR_NOMEM = 3,        /* workspace too small, or host allocation failed */
  TH_ERR_NOCONV = 4,       /* th_solve reached maxit before tol */
  TH_ERR_BREAKDOWN = 5,    /* Krylov breakdown (zero new direction before convergence) */
  TH_ERR_NONFINITE = 6,    /* NaN/Inf met in a residual norm */
  TH_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up */
  TH_ERR_UNSUPPORTED = 8,  /* valid but not implemented (e.g. Dirichlet sides in 3-D) */
  TH_ERR_SINGULAR = 9      /* a zero pivot during the FP64 set-up factorisations */
} th_status;

/* Boundary condition of one side (Section 2). */
/* Boundary condition per side (Section 2): Neumann (natural), absorbing
 * (Robin, -i k u), or Dirichlet (u = 0 on Gamma_0; 2-D, QSFEM coarse level):
 * the unknowns on Gamma_0 stay on the node grid and are decoupled by identity
 * rows and columns of the fine, subdomain and coarse operators, the coarse
 * space vanishes there too (the restriction gives 0 there and the
 * prolongation ignores those coarse values), so a right-hand side that is
 * zero on Gamma_0 gives a solution that is zero there. */
enum { TH_BC_NEUMANN = 0, TH_BC_ROBIN = 1, TH_BC_DIRICHLET = 2 };
/* Side index in th_mesh.bc: 0 = x low, 1 = x high, 2 = y low, 3 = y high. */

/* Storage / arithmetic precision of the two-grid cycle.
 *   TH_PREC_FP64: every step in FP64 (the plain form).
 *   TH_PREC_FP32, TH_PREC_BF16, TH_PREC_FP16: the cycle (operator applies,
 *   smoother, transfers, coarse solve) runs in FP32 complex arithmetic; the
 *   subdomain inverse rows are stored in FP32, BF16 or FP16 respectively and
 *   accumulated in FP32.  The FGMRES orthogonalisation, residual norms and its
 *   A z products stay FP64 in all modes; the set-up (inverse rows, QSFEM
 *   coefficients, coarse factorisation) is always computed in FP64. */
enum { TH_PREC_FP64 = 0, TH_PREC_FP32 = 1, TH_PREC_BF16 = 2, TH_PREC_FP16 = 3 };

/* Operators for th_apply. */
enum {
  TH_OP_A = 0,   /* fine Helmholtz matrix A (Eq. bilin_form) */
  TH_OP_AS = 1,  /* fine shifted matrix A_s: k^2 -> k^2 (1 + i alpha_s) (Section 4.1) */
  TH_OP_AQ = 2   /* coarse QSFEM matrix A_q (Section 3.3); x, y are coarse vectors */
};

typedef struct {
  int dim;      /* 2 (unit square) or 3 (unit cube; element order 2 only) */
  int n;        /* cells per direction, >= 1 */
  int p;        /* element order: 2, 4, 6 or 8 (2-D); 2 (3-D) */
  int bc[6];    /* TH_BC_* per side: x low, x high, y low, y high, z low, z high
                   (the z entries are ignored in 2-D) */
} th_mesh;

typedef struct {
  double alpha_s;   /* smoother shift (Section 4.1); the paper uses 0.2 */
  int l_dd;         /* subdomain size U^(i) in cells per direction (Section 4.5) */
  int n_dd;         /* DD iterations per smoother step (Algorithm 2), >= 1 */
  int n_s;          /* pre- and post-smoothing steps (Algorithm 1), >= 1 */
  double omega_c;   /* coarse-correction relaxation (Algorithm 1) */
  int prec;         /* active cycle precision, TH_PREC_* */
  unsigned prec_mask; /* additional precisions to prepare (bit 1 << TH_PREC_*),
                         so th_set_precision can switch without a new set-up */
  int restart;      /* FGMRES restart length m, >= 1 */
  int maxit;        /* FGMRES iteration limit */
  double tol;       /* relative residual target ||f - A u|| / ||f|| */
  int nrhs_max;     /* largest nrhs any later call will pass */
  int coarse_kind;  /* TH_CK_QSFEM: the QSFEM coarse operator of Section 3.3 on the
                       coarse grid of spacing 2h/p ('opt', the paper's method);
                       TH_CK_GALERKIN: standard Galerkin p-type coarsening of
                       Section 4 ('gal', the paper's comparison), A_c = I_P^T
                       A_{alpha_c} I_P = the Q_{p/2} operator on the same mesh
                       (2-D only; TH_ERR_UNSUPPORTED in 3-D) */
  double alpha_c;   /* TH_CK_GALERKIN: complex shift of the coarse operator's volume
                       term, k^2 (1 + i alpha_c) + i eps (Table 2); ignored for QSFEM */
  int coarse_chunks; /* 2-D QSFEM coarse solve: the number P of row chunks of its
                        partition (2 P - 1 <= m_c); 0 (the default) = round(sqrt(m_c)) */
} th_params;

enum { TH_CK_QSFEM = 0, TH_CK_GALERKIN = 1 };

typedef struct {
  int iters;            /* FGMRES iterations (max over right-hand sides) */
  int converged;        /* number of right-hand sides that met tol */
  double relres_max;    /* max over rhs of the true ||f - A u|| / ||f|| at exit */
  double ms_total;      /* wall time of th_solve (host clock, includes syncs) */
  int iters_per_rhs[64];/* iterations of the first min(nrhs, 64) right-hand sides */
  int fallbacks;        /* learned coarse corrector: restarts with the direct
                         * coarse solve (see th_set_coarse), else 0 */
} th_solve_info;

typedef struct th_ctx th_ctx;

/* ------------------------------------------------------------------ set-up */

/* Bytes of device workspace th_setup needs for this mesh and parameters.
 * Host-only computation.  Returns TH_ERR_ARG / TH_ERR_UNSUPPORTED for invalid
 * or unsupported inputs. */
th_status th_workspace_size(const th_mesh* mesh, const th_params* prm, size_t* bytes);

/* Builds a context: the FP64 set-up of Sections 3-4 (GLL reference matrices,
 * QSFEM cell coefficients, partition, subdomain inverse rows, coarse block
 * factorisation) on the host, then copies everything into `workspace_dev`.
 *   k_host, eps_host: double[n*n] per cell, row-major [cy][cx]; eps_host may
 *     be NULL (eps = 0).  Copied; the caller may free them after return.
 *   workspace_dev: device buffer of at least th_workspace_size bytes, 256-byte
 *     aligned, owned by the caller and kept alive until th_destroy.
 * Synchronous: returns after the copies have completed on `stream`. */
th_status th_setup(const th_mesh* mesh, const double* k_host, const double* eps_host,
                   const th_params* prm, void* workspace_dev, size_t bytes,
                   void* stream, th_ctx** out);

/* Device-side status: synchronises `stream` and returns TH_ERR_TIMEOUT if a
 * bounded device wait of an earlier kernel gave up (the flag is then cleared),
 * TH_OK otherwise.  Kernels that wait on mbarriers do so with an iteration
 * limit; on a timeout they drain their copies in flight and return early, so
 * the results of that launch are invalid. */
th_status th_device_status(th_ctx* ctx, void* stream);

/* Limit of every bounded device-side wait of the context's kernels (the
 * mbarrier waits of the streamed and tensor-core subdomain products, the
 * coarse chunk sweep's row exchange and the learned corrector's convolutions),
 * in polls of the barrier: polls < 0 restores each kernel's default (about a
 * second); polls > 0 sets that many; polls = 0 makes each such kernel record
 * a timeout (reported by th_device_status as TH_ERR_TIMEOUT) and return before
 * its first barrier, bulk copy or MMA, leaving its outputs unwritten.  The
 * last form exists to exercise the error path without stalling a GPU.  A
 * kernel that gives up still waits, with the default limit, for its own
 * copies and MMAs in flight before it returns.  Synchronous on `stream`. */
th_status th_set_wait_limit(th_ctx* ctx, long long polls, void* stream);

/* Selects the active cycle precision (must have been prepared at set-up). */
th_status th_set_precision(th_ctx* ctx, int prec);

/* Releases host-side state.  Does not touch the caller's workspace. */
void th_destroy(th_ctx* ctx);

const char* th_status_str(th_status s);

/* --------------------------------------------------------- hot-path steps */

/* y = OP x for nrhs right-hand sides (OP = A, A_s: fine vectors; A_q: coarse).
 * prec: TH_PREC_FP64 applies in FP64; TH_PREC_FP32 rounds x to FP32, applies
 * in FP32 and widens the result.  x and y must not overlap. */
th_status th_apply(th_ctx* ctx, int op, const double* x_dev, double* y_dev,
                   int nrhs, int prec, void* stream);

/* r = f - A u (the residual, fused with the apply), FP64. */
th_status th_residual(th_ctx* ctx, const double* f_dev, const double* u_dev,
                      double* r_dev, int nrhs, void* stream);

/* The mixed form's outer residual (the first step of th_cycle and th_smooth
 * when the active precision is not FP64): r = f - A u for FP64 f, u (layout as
 * th_residual), delivered rounded to FP32 in r (nrhs x N complex floats,
 * interleaved).  2-D: one kernel in double-single arithmetic (pairs of floats,
 * 48 significant bits; FP64 arithmetic is the scarce unit on this GPU), so r
 * carries the cancellation f - A u as the FP64 residual would; 3-D, or with
 * th_set_kernel_variant(TH_K_RESID, ., 0): the FP64 apply, then rounding.
 * TH_ERR_UNSUPPORTED when no FP32-cycle precision was prepared. */
th_status th_residual_mixed(th_ctx* ctx, const double* f, const double* u, float* r, int nrhs, void* stream);

/* One CSDDSmoother(u, f) step of Algorithm 2 in the active precision:
 * r = f - A u; v = 0; n_dd times DDStep(v, r; A_s); u += v.  Updates u. */
th_status th_smooth(th_ctx* ctx, const double* f_dev, double* u_dev, int nrhs, void* stream);

/* r_c = I_P^T r (restriction, the adjoint of the prolongation), FP64. */
th_status th_restrict(th_ctx* ctx, const double* r_dev, double* rc_dev, int nrhs, void* stream);

/* u += omega * I_P u_c (prolongation: degree-p/2 interpolation of the coarse
 * vertex values in every fine cell, Section 4.2), FP64. */
th_status th_prolong(th_ctx* ctx, const double* uc_dev, double* u_dev, double omega,
                     int nrhs, void* stream);

/* u_c = A_q^{-1} r_c: direct coarse solve with the FP64 block factorisation,
 * applied in the active precision. */
th_status th_coarse_solve(th_ctx* ctx, const double* rc_dev, double* uc_dev, int nrhs,
                          void* stream);

/* One TwoGridStep(u, f) of Algorithm 1 in the active precision; updates u.
 * With u = 0 on input it is the preconditioner of Section 4. */
th_status th_cycle(th_ctx* ctx, const double* f_dev, double* u_dev, int nrhs, void* stream);

/* th_cycle replayed from a CUDA graph (no counterpart in the paper; the
 * arithmetic is th_cycle's, bit for bit).  The first call for a given
 * (f_dev, u_dev, nrhs, active precision) captures th_cycle's kernel sequence
 * on a private stream of the context and instantiates it; that call and every
 * later call with the same arguments launch the graph on `stream`, so a cycle
 * costs one host call instead of about twenty kernel launches.  Captured
 * graphs hold the pointers they were captured with: the caller must keep
 * f_dev and u_dev valid (or stop calling with them).  th_set_precision and
 * th_set_kernel_variant invalidate the cache; at most 256 graphs are kept per
 * context (all are dropped when the cache is full).  While th_profile is on,
 * or after th_set_graphs(ctx, 0), it runs th_cycle directly.
 * Errors: those of th_cycle; TH_ERR_CUDA if capture or instantiation fails. */
th_status th_cycle_graph(th_ctx* ctx, const double* f_dev, double* u_dev, int nrhs, void* stream);

/* enable = 1 (default): th_cycle_graph and the preconditioner applications
 * inside th_solve replay captured graphs; enable = 0: they launch kernel by
 * kernel and the cached graphs are destroyed.  TH_ERR_ARG for other values. */
th_status th_set_graphs(th_ctx* ctx, int enable);

/* Same as th_cycle on host buffers: copies f and u to the device, runs the
 * cycle (as th_cycle_graph: replayed from a captured graph unless graphs are
 * off or profiling is on), copies u back; synchronous. */
th_status th_cycle_host(th_ctx* ctx, const double* f_host, double* u_host, int nrhs, void* stream);

/* th_coarse_solve without any workspace scratch (no counterpart in the paper).
 *
 * The same FP64 direct coarse solve u_c = A_q^{-1} r_c as th_coarse_solve on an
 * FP64-prepared context, for callers that cannot allocate device memory when
 * they need the solve: code running inside another framework's fixed memory
 * arena, allocation-free real-time paths, or a context shared read-only by
 * several users, none of whom may reserve per-call scratch.  Its scratch (the
 * forward-sweep block vectors) lives in a fixed 4 MiB device array of the
 * library, so the call uses only rc_dev (input), uc_dev (output) and the
 * context's factors, which it only reads.  It calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *   Scope: the 2-D dispersion-matched (QSFEM) coarse level of an FP64-prepared
 *   context.  3-D contexts, Galerkin-coarsened contexts and contexts without
 *   FP64 factors return TH_ERR_UNSUPPORTED.
 *   Limit: Nc * nrhs <= 262144 complex values (e.g. one right-hand side up to a
 *   401 x 401 coarse grid); larger requests return TH_ERR_ARG.  nrhs must not
 *   exceed the context's nrhs_max.  The current device must be the one the
 *   context was set up on (TH_ERR_ARG otherwise).
 *   The array is per GPU and stays allocated until the process exits.  Every
 *   call made outside a stream capture looks up the array's device address with
 *   the current device (so a device reset or another current context cannot
 *   leave a stale address); a call on a capturing stream reuses the address of
 *   the last uncaptured call on that device, so make one call on each device
 *   before capturing it, and none across a device reset inside a capture.
 *   All calls share the one array and it keeps the last call's contents (every
 *   entry is written before it is read, so nothing needs clearing); calls whose
 *   executions overlap on the GPU (other streams) race on it. */
th_status th_coarse_solve_noalloc(const th_ctx* ctx, const double* rc_dev, double* uc_dev, int nrhs,
                                  void* stream);

/* Right-preconditioned flexible GMRES(restart) with the two-grid
 * preconditioner, FP64 orthogonalisation.  u holds the initial guess on
 * input and the solution on output.  Synchronous (the Hessenberg update runs
 * on the host).  info may be NULL.  Returns TH_ERR_NOCONV if some right-hand
 * side has not reached tol within maxit (u then holds the last iterate). */
th_status th_solve(th_ctx* ctx, const double* f_dev, double* u_dev, int nrhs,
                   th_solve_info* info, void* stream);

/* th_solve on host buffers (copies in and out inside the call). */
th_status th_solve_host(th_ctx* ctx, const double* f_host, double* u_host, int nrhs,
                        th_solve_info* info, void* stream);

/* ---------------------------------------------------------------------------
 * Learned coarse corrector (no counterpart in the paper).
 *
 * A small convolutional U-Net on the coarse node grid that stands in for the
 * coarse solve "u_c = A_c^{-1} r_c" of Algorithm 1:
 *     u_c ~= s * UNet([Re r_c / s, Im r_c / s, eta]),  s = RMS(r_c),
 * eta = k h_c averaged from the coarse cells to the nodes (2-D only).  With L
 * levels and C_l = base * 2^l channels on the node grid zero-padded to a
 * multiple of 2^(L-1): per encoder level two 3x3 convolutions with SiLU and
 * 2x2 average pooling, per decoder level nearest doubling, concatenation
 * [skip, doubled] and two 3x3 convolutions with SiLU, then a 1x1 head to the
 * 2 output channels.  BF16 weights and activations, FP32 accumulation on the
 * tensor cores; FP32 master weights, gradients and Adam moments.
 * Parameters are FP32 arrays in this order, per convolution weights
 * [c_out][3][3][c_in] then bias [c_out]: encoder levels 0..L-1 (a, b), decoder
 * levels L-2..0 (a, b), head weights [2][base] and bias [2].
 * The network's buffers are allocated with cudaMalloc by th_unet_init (for
 * batch_max right-hand sides) and freed by th_destroy.
 * --------------------------------------------------------------------------- */

/* Number of FP32 parameters; TH_ERR_ARG unless levels in [2, 6], base a
 * multiple of 16, base 2^(L-1) <= 256 and 3 base 2^(L-2) <= 256. */
th_status th_unet_param_count(int levels, int base, size_t* n);

/* Creates (or replaces) the context's corrector with the given initial
 * parameters (host, n = th_unet_param_count).  Synchronous.
 * TH_ERR_UNSUPPORTED for a 3-D context, TH_ERR_NOMEM if allocation fails. */
th_status th_unet_init(th_ctx* ctx, int levels, int base, int batch_max, const float* params_host,
                       size_t n, void* stream);

/* Copies the FP32 master parameters to / from the host (synchronous); a set
 * also resets the Adam state. */
th_status th_unet_get_params(th_ctx* ctx, float* params_host, size_t n, void* stream);
th_status th_unet_set_params(th_ctx* ctx, const float* params_host, size_t n, void* stream);

/* The network alone (for checks): in [batch][mp][mp][3] FP32 (padded node
 * grid, mp = the node count rounded up to a multiple of 2^(L-1)) ->
 * out [batch][mp][mp][2] FP32; batch <= batch_max. */
th_status th_unet_forward(th_ctx* ctx, const float* in_dev, float* out_dev, int batch, void* stream);

/* Gradients of sum(out * gout) with respect to every parameter (FP32, the
 * parameter order above) for the activations of the last th_unet_forward. */
th_status th_unet_backward(th_ctx* ctx, const float* gout_dev, float* grads_dev, int batch,
                           void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * loss mean_b ||out_b - u_b / s_b||^2 / ||u_b / s_b||^2 over the unpadded
 * nodes for pairs (r_c, u_c) in FP64 complex [batch][N_c] on the device;
 * *loss (may be NULL) receives the loss before the step (synchronous then). */
th_status th_unet_train_step(th_ctx* ctx, const double* rc_dev, const double* uc_dev, int batch,
                             double lr, double* loss, void* stream);

/* u_c = s UNet(r_c / s) for nrhs coarse residuals (FP64 complex [nrhs][N_c]). */
th_status th_unet_correct(th_ctx* ctx, const double* rc_dev, double* uc_dev, int nrhs, void* stream);

/* Coarse correction inside th_cycle / th_solve: TH_COARSE_DIRECT (default),
 * TH_COARSE_LEARNED (needs th_unet_init) or TH_COARSE_NONE (u_c = 0: the
 * smoother alone, for comparison).  With TH_COARSE_LEARNED and plain_iters >
 * 0, th_solve switches to the direct solve (restarting from its current
 * iterate) once its iteration count reaches ceil(1.5 plain_iters), and counts
 * that in th_solve_info.fallbacks; plain_iters = 0 disables the fallback. */
enum { TH_COARSE_DIRECT = 0, TH_COARSE_LEARNED = 1, TH_COARSE_NONE = 2 };
th_status th_set_coarse(th_ctx* ctx, int mode, int plain_iters);

/* Number of kernel launches the library issued since the context was built
 * (all entry points), for accounting. */
th_status th_launch_count(const th_ctx* ctx, long long* launches);

/* Kernel classes for th_profile_read. */
enum {
  TH_K_FINE = 0,        /* fine operator apply / residual (K1, K2) */
  TH_K_DD = 1,          /* subdomain inverse-row products (K3) */
  TH_K_COMBINE = 2,     /* interface averaging and update (K4) */
  TH_K_RESTRICT = 3,    /* restriction (K5) */
  TH_K_PROLONG = 4,     /* prolongation and correction (K6) */
  TH_K_COARSE_APPLY = 5,/* coarse QSFEM apply (K7) */
  TH_K_COARSE_SOLVE = 6,/* coarse block-tridiagonal solve (K8) */
  TH_K_VECTOR = 7,      /* precision conversions, axpy, zero fill (K10) */
  TH_K_KRYLOV = 8,      /* FGMRES dots, norms, updates (K9) */
  TH_K_COUNT = 9,
  TH_K_DD_BATCH = 9,    /* (variants only) batched BF16 subdomain products: 0 CUDA cores, 1 tensor cores */
  TH_K_RESID = 10,      /* (variants only) the mixed form's outer residual, see th_residual_mixed */
  TH_K_CYCLE = 11,      /* (variants only) launch structure of the cycle, see th_set_kernel_variant */
  TH_K_COARSE_MULTI = 12, /* (variants only) 2-D coarse sweep for 8 or more right-hand sides */
  TH_K_AZ = 13,         /* (variants only) the FGMRES product A z of the mixed forms */
  TH_K_COARSE_REFINE = 14, /* (variants only) refinement steps of the mixed 2-D coarse solve */
  TH_K_SEP_SYM = 15     /* (variants only) one-rhs FP32 separator product from Sinv's upper triangle */
};

/* Per-kernel timing for measurement: with enable = 1 every later kernel
 * launch of the context is bracketed by two CUDA events recorded on the
 * stream it is launched on (previous records are discarded); enable = 0 stops
 * recording.  Records beyond an internal pool of 65536 launches are dropped. */
th_status th_profile(th_ctx* ctx, int enable);

/* Sum of the event-timed durations (ms) and the number of launches of kernel
 * class `kind` since th_profile(ctx, 1).  Synchronises on the recorded events. */
th_status th_profile_read(th_ctx* ctx, int kind, double* ms, long long* launches);

/* Arithmetic peak probe (measurement only; no counterpart in the paper):
 * the FMA rate of the FP64 (prec = TH_PREC_FP64) or FP32 (TH_PREC_FP32)
 * pipe of the current device, in flop/s (2 per fused multiply-add), from
 * 8 blocks of 256 threads per SM each running 8 independent chains of `iters`
 * dependent FMAs, timed with CUDA events on `stream` after one shorter
 * warm-up launch.  Synchronous.  The roofline of kernels bound by these pipes
 * (the FP64 form's subdomain products, the double-single residual) is taken
 * against this rate.  TH_ERR_ARG for another prec or iters < 1. */
th_status th_peak_fma(int prec, int iters, double* flops_per_s, void* stream);

/* Kernel variants chosen by the set-up autotuner (which times each candidate
 * on the context's own problem with CUDA events):
 *   TH_K_FINE: 0 = large cell tile, 1 = small cell tile (the set-up times both
 *              for one right-hand side and, with nrhs_max >= 8, for nrhs_max, per
 *              precision; setting a variant sets it for every right-hand-side count,
 *              and prec FP32 also sets the double-single apply's);
 *   TH_K_DD:   0 = per-subdomain CTAs with direct loads,
 *              1 = persistent CTAs streaming the rows through TMA bulk copies,
 *              2 = the same with a dedicated producer warp and per-slot
 *                  mbarrier release (no CTA barrier per ring slot; the
 *                  autotuner's usual choice for one rhs on BF16 rows),
 *              3 = variant 1 with smaller ring stages, three CTAs per SM,
 *              4, 5 = variants 1, 3 with paired FP32 FMAs (FP32 cycle on
 *                  BF16 / FP16 rows only; prec must be TH_PREC_FP32; on FP32
 *                  rows they run variants 1, 3);
 *   TH_K_DD_BATCH: 1 (default when the BF16 rows fit, U box <= 128 nodes) runs
 *              the products of 8 or more right-hand sides on the tensor cores
 *              (tcgen05.mma, BF16 operands, FP32 accumulation; the residuals
 *              are rounded to BF16), 0 keeps them on the CUDA cores;
 *   TH_K_RESID: 1 (default) double-single residual kernel, 0 FP64 apply and
 *              rounding (th_residual_mixed; prec is ignored);
 *   TH_K_CYCLE: 1 (default) a TwoGridStep with u = 0 on entry (the
 *              preconditioner, and the mixed form's inner step) of a 2-D
 *              context with n_s = n_dd = 1 folds the RAS-like average into
 *              the next fine apply, the prolongation and correction into the
 *              post-smoother's fine apply, and the last average, the update
 *              and (mixed form) the widening to FP64 into one kernel: the
 *              same arithmetic in the same order as 0, the step-by-step
 *              launches (prec is ignored); 2 = 1 with every launch after the
 *              first issued with a programmatic dependency on the one before
 *              (it may be scheduled while that one drains, and waits for it
 *              before touching shared data; not while th_profile records);
 *   TH_K_AZ:   the product w = A z of each FGMRES step in the mixed forms
 *              (2-D): 1 (default) the double-single apply with FP64 output
 *              (48-bit significands; the final residual is still recomputed
 *              with the FP64 apply), 0 the FP64 apply; prec is ignored;
 *   TH_K_COARSE_MULTI: the 2-D coarse chunk sweep for 8 or more right-hand
 *              sides: 1 (default) one CTA per chunk and group of 8 to 16
 *              right-hand sides (the narrowest group that keeps the chunks x
 *              groups within one CTA per SM), each G_j streamed once for all
 *              groups through L2; 0 one
 *              thread-block cluster per chunk and tile of 2-8 right-hand sides
 *              (the tile count multiplies the G_j reads); 2 the column-group
 *              sweep of variant 1, then the separator product and the spike
 *              correction on the tensor cores for groups of up to 64
 *              right-hand sides, with the reduced inverse, the spikes and
 *              their operands each held as two BF16 numbers (hi + lo, 16
 *              significant bits; mixed contexts with nrhs_max >= 8, else as
 *              variant 1); prec is ignored;
 *   TH_K_KRYLOV: the FGMRES Gram-Schmidt dots, norms and updates of the
 *              mixed forms: 1 (default) double-single arithmetic on the FP64
 *              vectors (exact two-float splits, products with their exact
 *              rounding errors, compensated sums: about 2^-44 relative),
 *              0 FP64; the FP64 form always uses FP64; prec is ignored;
 *   TH_K_SEP_SYM: the one-right-hand-side FP32 separator product of the 2-D
 *              coarse solve: 1 (default) from the upper triangle of the
 *              complex-symmetric reduced inverse only (64 x 64 blocks, each
 *              serving S_IJ x_J and S_IJ^T x_I; half the bytes), 0 the full
 *              GEMV; prec is ignored;
 *   TH_K_COARSE_REFINE: steps (0 to 3) of iterative refinement after the
 *              mixed form's 2-D coarse solve: z = r_c - A_q u_c in FP32, the
 *              same solve of z, u_c += its solution.  The set-up chooses the
 *              default from the FP32 solve's residual on a seeded right-hand
 *              side; prec is ignored;
 *   TH_K_COARSE_SOLVE: one-right-hand-side chunk sweep of the 2-D coarse
 *              solve: 0 = two phases per block step (512 threads), 1 = one
 *              cluster barrier per step (1024 threads, m_c <= 256), 2 = rows
 *              exchanged by st.async on per-slot mbarriers, no cluster
 *              barrier per step (1024 threads, m_c <= 256; bounded waits
 *              report through th_device_status).
 * prec selects the FP64 or the FP32-cycle kernels (TH_PREC_FP64 / TH_PREC_FP32).
 * Overriding is for testing and measurement; every variant computes the same
 * result up to summation order. */
th_status th_set_kernel_variant(th_ctx* ctx, int kernel, int prec, int variant);
th_status th_get_kernel_variant(const th_ctx* ctx, int kernel, int prec, int* variant);

/* ------------------------------------------------- host-side set-up data */
/* These run on the host only (no GPU needed) and expose the FP64 set-up the
 * device path is built from, so that it can be checked on its own. */

/* 1-D reference matrices of Q_p on [0,1] with the GLL Lagrange basis:
 * nodes[p+1], mass[(p+1)^2], stiff[(p+1)^2] (row-major), integrated exactly. */
th_status th_host_reference_1d(int p, double* nodes, double* mass, double* stiff);

/* QSFEM per-cell coefficients (Section 3.3) of one coarse cell of size hc with
 * wavenumber k and damping eps: out[6] = (d0, d1, d2) complex interleaved,
 * d0 = N P0/4 - i eps hc^2/9, d1 = N P1/2 - i eps hc^2/18, d2 = N P2 - i eps hc^2/36. */
th_status th_host_qsfem_cell(double k, double eps, double hc, double* out);

/* Inverse rows of one subdomain matrix A_s^(i) (Algorithm 2) of the mesh
 * (as th_setup would build them): subdomain index `sub` in the row-major
 * block order; out receives rows x cols complex values (interleaved FP64),
 * row r = U-box dof r (lexicographic in the U box), column c = Omega-box dof
 * c, scaled by 1/L_j, where the boxes are given as
 * box[12] = (ox, oy, wx, wy, ux, uy, vx, vy, oz, wz, uz, vz) in global dof
 * coordinates (Omega origin and widths, U origin and widths; in 2-D oz = uz
 * = 0 and wz = vz = 1).  out receives Lu^d x Lw^d complex values. */
/* The four pair weights of one coarse cell of the 3-D coarse operator (the
 * project's fitted 27-point scheme, the 3-D counterpart of Eq. P_QSFEM and
 * Eq. element_wise_qsfem): out[2 i], out[2 i + 1] = Re, Im of
 * h_c N P_i w_i - i eps h_c^3 (1/3)^(3-i) (1/6)^i, i = number of coordinates
 * in which the two vertices differ, w = (1/8, 1/4, 1/2, 1).  Host only. */
th_status th_host_qsfem27_cell(double k, double eps, double hc, double* out);

th_status th_host_inverse_rows(const th_mesh* mesh, const double* k_host, const double* eps_host,
                               const th_params* prm, int sub, int* box, double* out,
                               size_t out_len);

/* Host-only probe of the Galerkin p-type coarse set-up (Section 4; 2-D,
 * prm->coarse_kind ignored, prm->alpha_c used).  Writes the coarse operator as
 * a (2q+1)^2-point stencil per coarse node, q = p/2, interleaved complex:
 * stencil[((y mc + x) (2q+1) + dy + q) (2q+1) + dx + q] = A_c[(y, x), (y+dy, x+dx)]
 * (stencil_len doubles, at least 2 mc^2 (2q+1)^2).  If b and x are non-NULL,
 * also solves A_c x = b (mc^2 complex each) with the block sweep of the FP64
 * block inverses the device solve uses.  TH_ERR_NOMEM if stencil_len is short. */
th_status th_host_galerkin(const th_mesh* mesh, const double* k_host, const double* eps_host,
                           const th_params* prm, double* stencil, size_t stencil_len,
                           const double* b, double* x);

/* Host-only probe of the partitioned coarse set-up (Algorithm 1's coarse solve,
 * 2-D QSFEM coarse level): with the coarse node rows split into P chunks and
 * P - 1 separator rows, writes the separator row indices (sep, P - 1 ints)
 * and the explicit inverse of the reduced separator system that the device
 * solve applies, sinv[((k mc + r) (P-1) mc + k' mc + r')] (interleaved
 * complex, row-major, (P-1) mc square; sinv_len doubles, at least
 * 2 ((P-1) mc)^2).  That matrix is the separator block of A_q^{-1}.
 * TH_ERR_ARG unless 2 <= P and 2P - 1 <= mc; TH_ERR_NOMEM if sinv_len is short. */
th_status th_host_coarse_separators(const th_mesh* mesh, const double* k_host, const double* eps_host,
                                    const th_params* prm, int P, int* sep, double* sinv, size_t sinv_len);

/* ---------------------------------------------------- Fourier analysis */

/* Dispersion error of a compact 2-D stencil (Section 3.2): for a symmetric
 * 3 x 3 stencil P with symbol sigma_P(xi) (Eq. symbol_sigma_P) on the grid of
 * spacing h and eta = k h, the distance of its zero set Z_P to the circle
 * |xi| = k,
 *     D_P = max_{t in [-pi, pi]} min_{xi in Z_P} |k (cos t, sin t) - xi| ,
 * returned divided by k, over the directions t_j = -pi + 2 pi j / nt.
 *   kind: TH_DISP_QSFEM (Eq. P_QSFEM, from the same cancellation-free weights as
 *         the coarse operator), TH_DISP_Q1 (bilinear elements: stiffness minus
 *         eta^2 times mass, Section 3.3), TH_DISP_FD5 (5-point differences).
 *   eta: host, n values in (0, 2];  d_max: host, n values (output);
 *   d_theta: host, n x nt values (output, index i nt + j) or NULL.
 * One GPU thread per (eta, t_j), FP64: the zero along each ray by a sign-change
 * scan and bisection, the nearest point by a scan over nearby rays and a
 * golden-section search.  Allocates and frees its own device buffers;
 * synchronous on `stream`.  TH_ERR_ARG for invalid arguments. */
enum { TH_DISP_QSFEM = 0, TH_DISP_Q1 = 1, TH_DISP_FD5 = 2 };
th_status th_dispersion(int kind, const double* eta, int n, int nt, double* d_max, double* d_theta, void* stream);

/* Local Fourier analysis of the two-grid method (Section 6, Eq. symbol_sum):
 * for nparam parameter points on the periodic plane with constant k and eps
 * (Q_p, p in {2, 4, 6}; coarse level TH_CK_QSFEM, or TH_CK_GALERKIN with
 * A_c = I_R A_{alpha_c} I_P (Section 4, Fig. 3 (a)); the exact shifted smoother
 * S = I - A_s^{-1} A), the spectral radius of the Bloch symbol
 * M(theta) = S^{n_s} K S^{n_s}, K = I - omega_c I_P A_c^{-1} I_R A, on the
 * grid theta = (-pi + 2 pi i / npts, -pi + 2 pi j / npts), and its maximum.
 *   params: host, nparam x 4 doubles (k h, eps / k^2, alpha_s, omega_c), k h > 0.
 *   rho_max: host, nparam doubles (output): the maximum over the grid.
 *   rho_theta: host, nparam x npts^2 doubles (output, index i npts + j), or NULL.
 * The symbols' blocks are assembled on the host in FP64; one CTA per
 * (parameter point, theta) forms the symbols, eliminates, and evaluates rho by
 * Gelfand's formula with 40 normalised squarings (relative error ~1e-10).
 * Allocates and frees its own device buffers; synchronous on `stream`.
 * TH_ERR_ARG for invalid sizes or parameters, TH_ERR_UNSUPPORTED for other p. */
th_status th_lfa_rho(int p, int n_s, int npts, int coarse_kind, double alpha_c, const double* params, int nparam,
                     double* rho_max, double* rho_theta, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TH_H */
