"""GB300 two-grid Helmholtz solver (arXiv 2509.17494): Python binding of include/th.h.

Argument marshalling only: every step of the solver runs in the native
library libth.so (hand-written sm_103a CUDA kernels plus the FP64 host
set-up).  PyTorch provides device memory and streams.  If the library is
missing the binding raises; there is no fallback implementation.

Vectors are torch.complex128 CUDA tensors of shape (N,) or (nrhs, N) with
N = (n p + 1)^2 (fine) or Nc = (n p / 2 + 1)^2 (coarse), lexicographic node
order with x fastest.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["TwoGridSolver", "lib", "library_path", "workspace_size", "host_reference_1d",
           "host_qsfem_cell", "host_inverse_rows", "PREC", "OPS", "ThError"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libth.so")
_LIB = None

PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}
OPS = {"A": 0, "As": 1, "Aq": 2}
BC = {"neumann": 0, "robin": 1, "dirichlet": 2}
SIDES = ("xlo", "xhi", "ylo", "yhi", "zlo", "zhi")


class ThError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {lib().th_status_str(code).decode()} (status {code})")


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("p", ctypes.c_int), ("bc", ctypes.c_int * 6)]


class Params(ctypes.Structure):
    _fields_ = [("alpha_s", ctypes.c_double), ("l_dd", ctypes.c_int), ("n_dd", ctypes.c_int),
                ("n_s", ctypes.c_int), ("omega_c", ctypes.c_double), ("prec", ctypes.c_int),
                ("prec_mask", ctypes.c_uint), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("tol", ctypes.c_double), ("nrhs_max", ctypes.c_int), ("coarse_kind", ctypes.c_int),
                ("alpha_c", ctypes.c_double), ("coarse_chunks", ctypes.c_int)]


COARSE_KIND = {"qsfem": 0, "gal": 1}   # TH_CK_QSFEM ('opt', Section 3.3), TH_CK_GALERKIN ('gal', Section 4)


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("relres_max", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("iters_per_rhs", ctypes.c_int * 64), ("fallbacks", ctypes.c_int)]


def library_path() -> str:
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    """Loads libth.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(there is no non-native fallback)")
    L = ctypes.CDLL(_LIB_PATH)
    P, I, D, U, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint, None
    sig = {
        "th_status_str": ([I], ctypes.c_char_p),
        "th_workspace_size": ([ctypes.POINTER(Mesh), ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)], I),
        "th_setup": ([ctypes.POINTER(Mesh), P, P, ctypes.POINTER(Params), P, ctypes.c_size_t, P,
                      ctypes.POINTER(P)], I),
        "th_set_precision": ([P, I], I),
        "th_device_status": ([P, P], I),
        "th_set_kernel_variant": ([P, I, I, I], I),
        "th_get_kernel_variant": ([P, I, I, ctypes.POINTER(I)], I),
        "th_destroy": ([P], V),
        "th_apply": ([P, I, P, P, I, I, P], I),
        "th_residual": ([P, P, P, P, I, P], I),
        "th_residual_mixed": ([P, P, P, P, I, P], I),
        "th_smooth": ([P, P, P, I, P], I),
        "th_restrict": ([P, P, P, I, P], I),
        "th_prolong": ([P, P, P, D, I, P], I),
        "th_coarse_solve": ([P, P, P, I, P], I),
        "th_cycle": ([P, P, P, I, P], I),
        "th_cycle_graph": ([P, P, P, I, P], I),
        "th_unet_param_count": ([I, I, ctypes.POINTER(ctypes.c_size_t)], I),
        "th_unet_init": ([P, I, I, I, P, ctypes.c_size_t, P], I),
        "th_unet_get_params": ([P, P, ctypes.c_size_t, P], I),
        "th_unet_set_params": ([P, P, ctypes.c_size_t, P], I),
        "th_unet_forward": ([P, P, P, I, P], I),
        "th_unet_backward": ([P, P, P, I, P], I),
        "th_unet_train_step": ([P, P, P, I, D, ctypes.POINTER(ctypes.c_double), P], I),
        "th_unet_correct": ([P, P, P, I, P], I),
        "th_set_coarse": ([P, I, I], I),
        "th_set_graphs": ([P, I], I),
        "th_cycle_host": ([P, P, P, I, P], I),
        "th_solve": ([P, P, P, I, ctypes.POINTER(SolveInfo), P], I),
        "th_solve_host": ([P, P, P, I, ctypes.POINTER(SolveInfo), P], I),
        "th_launch_count": ([P, ctypes.POINTER(ctypes.c_longlong)], I),
        "th_set_wait_limit": ([P, ctypes.c_longlong, P], I),
        "th_peak_fma": ([I, I, ctypes.POINTER(ctypes.c_double), P], I),
        "th_dispersion": ([I, P, I, I, P, P, P], I),
        "th_profile": ([P, I], I),
        "th_profile_read": ([P, I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)], I),
        "th_host_reference_1d": ([I, P, P, P], I),
        "th_host_qsfem_cell": ([D, D, D, P], I),
        "th_host_qsfem27_cell": ([D, D, D, P], I),
        "th_host_inverse_rows": ([ctypes.POINTER(Mesh), P, P, ctypes.POINTER(Params), I, P, P,
                                  ctypes.c_size_t], I),
        "th_host_galerkin": ([ctypes.POINTER(Mesh), P, P, ctypes.POINTER(Params), P, ctypes.c_size_t, P, P], I),
        "th_host_coarse_separators": ([ctypes.POINTER(Mesh), P, P, ctypes.POINTER(Params), I, P, P,
                                       ctypes.c_size_t], I),
        "th_lfa_rho": ([I, I, I, I, D, P, I, P, P, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = L
    return L


def _check(code, what):
    if code != 0:
        raise ThError(code, what)


def _mesh(n, p, bc, dim=2):
    m = Mesh()
    m.dim, m.n, m.p = int(dim), int(n), int(p)
    if isinstance(bc, str):
        vals = [BC[bc]] * 6
    else:
        vals = [BC[bc.get(s, "neumann")] for s in SIDES]
    for i, v in enumerate(vals):
        m.bc[i] = v
    return m


def _params(alpha_s=0.5, l_dd=2, n_dd=1, n_s=1, omega_c=1.0, prec="fp64", extra_prec=(), restart=30,
            maxit=200, tol=1e-8, nrhs_max=1, coarse="qsfem", alpha_c=0.0, coarse_chunks=0):
    q = Params()
    q.alpha_s, q.l_dd, q.n_dd, q.n_s, q.omega_c = float(alpha_s), int(l_dd), int(n_dd), int(n_s), float(omega_c)
    q.prec = PREC[prec]
    mask = 0
    for e in extra_prec:
        mask |= 1 << PREC[e]
    q.prec_mask = mask
    q.restart, q.maxit, q.tol, q.nrhs_max = int(restart), int(maxit), float(tol), int(nrhs_max)
    q.coarse_kind, q.alpha_c = COARSE_KIND[coarse], float(alpha_c)
    q.coarse_chunks = int(coarse_chunks)
    return q


def unet_param_shapes(levels=4, base=16):
    """(name, shape) of the corrector's parameters in the library's order (see th.h)."""
    C = [base << l for l in range(levels)]
    out, prev = [], 3
    for l in range(levels):
        out += [(f"e{l}a.w", (C[l], 3, 3, prev)), (f"e{l}a.b", (C[l],)),
                (f"e{l}b.w", (C[l], 3, 3, C[l])), (f"e{l}b.b", (C[l],))]
        prev = C[l]
    for l in range(levels - 2, -1, -1):
        out += [(f"d{l}a.w", (C[l], 3, 3, C[l] + C[l + 1])), (f"d{l}a.b", (C[l],)),
                (f"d{l}b.w", (C[l], 3, 3, C[l])), (f"d{l}b.b", (C[l],))]
    return out + [("head.w", (2, C[0])), ("head.b", (2,))]


def unet_param_count(levels=4, base=16) -> int:
    """FP32 parameter count of the learned coarse corrector (th_unet_param_count)."""
    n = ctypes.c_size_t(0)
    _check(lib().th_unet_param_count(int(levels), int(base), ctypes.byref(n)), "th_unet_param_count")
    return n.value


def workspace_size(n, p, bc="robin", **params) -> int:
    out = ctypes.c_size_t(0)
    dim = params.pop("dim", 2)
    m, q = _mesh(n, p, bc, dim), _params(**params)
    _check(lib().th_workspace_size(ctypes.byref(m), ctypes.byref(q), ctypes.byref(out)), "th_workspace_size")
    return out.value


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def host_reference_1d(p):
    nodes, M, K = np.zeros(p + 1), np.zeros((p + 1) ** 2), np.zeros((p + 1) ** 2)
    _check(lib().th_host_reference_1d(p, nodes.ctypes.data, M.ctypes.data, K.ctypes.data), "th_host_reference_1d")
    return nodes, M.reshape(p + 1, p + 1), K.reshape(p + 1, p + 1)


def host_qsfem_cell(k, eps, hc):
    out = np.zeros(6)
    _check(lib().th_host_qsfem_cell(float(k), float(eps), float(hc), out.ctypes.data), "th_host_qsfem_cell")
    return out[0::2] + 1j * out[1::2]


def host_qsfem27_cell(k, eps, hc):
    """The 4 complex pair weights of one coarse cell of the 3-D coarse operator."""
    out = np.zeros(8)
    _check(lib().th_host_qsfem27_cell(float(k), float(eps), float(hc), out.ctypes.data), "th_host_qsfem27_cell")
    return out[0::2] + 1j * out[1::2]


def host_inverse_rows(n, p, k_cell, eps_cell, sub, bc="robin", **params):
    """(box, W) of subdomain `sub` as the set-up computes it on the host."""
    dim = params.pop("dim", 2)
    m, q = _mesh(n, p, bc, dim), _params(**params)
    k, kp = _f64(k_cell)
    e, ep = _f64(eps_cell if eps_cell is not None else np.zeros_like(k))
    l_dd = max(1, min(int(params.get("l_dd", 2)), n))
    # maximal U / Omega box widths
    nb = -(-n // l_dd)
    lmax = -(-n // nb)
    Lu = lmax * p + 1
    Lw = min(lmax + 2, n) * p + 1
    out = np.zeros(2 * Lu ** dim * Lw ** dim)
    box = (ctypes.c_int * 12)()
    _check(lib().th_host_inverse_rows(ctypes.byref(m), kp, ep, ctypes.byref(q), int(sub), box, out.ctypes.data,
                                      out.size), "th_host_inverse_rows")
    W = (out[0::2] + 1j * out[1::2]).reshape(Lu ** dim, Lw ** dim)
    return list(box), W, Lu, Lw


def host_galerkin(n, p, k_cell, eps_cell=None, bc="robin", alpha_c=0.0, b=None):
    """(stencil, x) of the host Galerkin coarse set-up: stencil[(y, x), dy + q, dx + q]
    = A_c[(y, x), (y + dy, x + dx)], and x = A_c^{-1} b by the host block sweep if b is given."""
    q = p // 2
    mc = n * q + 1
    S = 2 * q + 1
    m, prm = _mesh(n, p, bc, 2), _params(alpha_c=alpha_c)
    k, kp = _f64(k_cell)
    e, ep = _f64(eps_cell if eps_cell is not None else np.zeros_like(k))
    st = np.zeros(2 * mc * mc * S * S)
    bp = xp = None
    if b is not None:
        bb = np.ascontiguousarray(np.asarray(b, dtype=np.complex128).reshape(-1))
        xo = np.zeros(mc * mc, dtype=np.complex128)
        bp, xp = bb.ctypes.data, xo.ctypes.data
    _check(lib().th_host_galerkin(ctypes.byref(m), kp, ep, ctypes.byref(prm), st.ctypes.data, st.size, bp, xp),
           "th_host_galerkin")
    sten = (st[0::2] + 1j * st[1::2]).reshape(mc * mc, S, S)
    return sten, (xo if b is not None else None)


def dispersion(kind, eta, nt=64, per_theta=False, stream=None):
    """D_P / k (Section 3.2) of the 'qsfem', 'q1' or 'fd5' stencil at each eta = k h, on the
    GPU (th_dispersion): max over nt directions, and the per-direction values if asked."""
    e = np.ascontiguousarray(np.atleast_1d(np.asarray(eta, dtype=np.float64)))
    dmax = np.zeros(e.size)
    dt = np.zeros((e.size, nt)) if per_theta else None
    k = {"qsfem": 0, "q1": 1, "fd5": 2}[kind]
    st = ctypes.c_void_p(stream) if stream is not None else None
    _check(lib().th_dispersion(k, e.ctypes.data, e.size, int(nt), dmax.ctypes.data,
                               dt.ctypes.data if per_theta else None, st), "th_dispersion")
    return (dmax, dt) if per_theta else dmax


def peak_fma(prec="fp64", iters=None, stream=None):
    """Measured FMA rate of the FP64 or FP32 pipe of the current device, flop/s."""
    if iters is None:
        iters = 4096 if prec == "fp64" else 262144
    v = ctypes.c_double(0)
    st = ctypes.c_void_p(stream) if stream is not None else None
    _check(lib().th_peak_fma(PREC[prec], int(iters), ctypes.byref(v), st), "th_peak_fma")
    return v.value


def host_coarse_separators(n, p, k_cell, eps_cell=None, bc="robin", P=3):
    """(separator rows, explicit inverse of the reduced separator system) of the
    host partitioned coarse set-up with P chunks (th_host_coarse_separators)."""
    mc = n * p // 2 + 1
    nred = (P - 1) * mc
    m, prm = _mesh(n, p, bc, 2), _params()
    k, kp = _f64(k_cell)
    e, ep = _f64(eps_cell if eps_cell is not None else np.zeros_like(k))
    sep = np.zeros(P - 1, dtype=np.int32)
    out = np.zeros(2 * nred * nred)
    _check(lib().th_host_coarse_separators(ctypes.byref(m), kp, ep, ctypes.byref(prm), int(P), sep.ctypes.data,
                                           out.ctypes.data, out.size), "th_host_coarse_separators")
    return sep, (out[0::2] + 1j * out[1::2]).reshape(nred, nred)


def lfa_rho(p, params, n_s=1, npts=48, per_theta=False, coarse="qsfem", alpha_c=0.0, stream=None):
    """Fourier analysis of the two-grid method on the GPU (th_lfa_rho).

    params: (nparam, 4) array of (k h, eps / k^2, alpha_s, omega_c).  Returns the
    maximum of rho(M(theta)) over the npts x npts theta grid per parameter point,
    and with per_theta also the (nparam, npts, npts) values."""
    prm = np.ascontiguousarray(np.atleast_2d(np.asarray(params, dtype=np.float64)))
    if prm.shape[1] != 4:
        raise ValueError("params must have 4 columns (k h, eps / k^2, alpha_s, omega_c)")
    nparam = prm.shape[0]
    rmax = np.zeros(nparam)
    rth = np.zeros((nparam, npts, npts)) if per_theta else None
    _check(lib().th_lfa_rho(int(p), int(n_s), int(npts), COARSE_KIND[coarse], float(alpha_c), prm.ctypes.data, nparam,
                            rmax.ctypes.data, rth.ctypes.data if per_theta else None, stream), "th_lfa_rho")
    return (rmax, rth) if per_theta else rmax


class TwoGridSolver:
    """A set-up context of the two-grid preconditioned FGMRES solver on one GPU."""

    def __init__(self, n, p, k_cell, eps_cell=None, bc="robin", alpha_s=0.5, l_dd=2, n_dd=1, n_s=1,
                 omega_c=1.0, prec="fp64", extra_prec=(), restart=30, maxit=200, tol=1e-8, nrhs_max=1,
                 device=None, dim=None, coarse="qsfem", alpha_c=0.0, coarse_chunks=0):
        """coarse: 'qsfem' (the QSFEM coarse operator, the paper's 'opt') or 'gal'
        (standard Galerkin p-type coarsening with coarse shift alpha_c, 2-D);
        coarse_chunks: row chunks of the 2-D coarse partition (0: round(sqrt(m_c)))."""
        import torch

        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("TwoGridSolver needs a CUDA device (no CPU fallback)")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.n, self.p = int(n), int(p)
        kshape = np.shape(k_cell)
        self.dim = int(dim) if dim is not None else (3 if len(kshape) == 3 else 2)
        self.N = (self.n * self.p + 1) ** self.dim
        self.Nc = (self.n * self.p // 2 + 1) ** self.dim
        self.nrhs_max = int(nrhs_max)
        self._mesh = _mesh(n, p, bc, self.dim)
        self._params = _params(alpha_s, l_dd, n_dd, n_s, omega_c, prec, extra_prec, restart, maxit, tol, nrhs_max,
                               coarse, alpha_c, coarse_chunks)
        self.coarse_kind = coarse
        L = lib()
        nb = ctypes.c_size_t(0)
        _check(L.th_workspace_size(ctypes.byref(self._mesh), ctypes.byref(self._params), ctypes.byref(nb)),
               "th_workspace_size")
        self.workspace_bytes = nb.value
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        self._k, kp = _f64(np.asarray(k_cell, dtype=float).reshape(-1))
        if eps_cell is None:
            ep = None
        else:
            self._e, ep = _f64(np.asarray(eps_cell, dtype=float).reshape(-1))
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = L.th_setup(ctypes.byref(self._mesh), kp, ep, ctypes.byref(self._params),
                            ctypes.c_void_p(self.workspace.data_ptr()), nb.value, self._stream(),
                            ctypes.byref(ctx))
        _check(st, "th_setup")
        self._ctx = ctx

    # ------------------------------------------------------------- helpers
    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream)

    def _vec(self, t, length, name):
        torch = self.torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or t.device != self.device:
            raise TypeError(f"{name} must be a complex128 tensor on {self.device}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() % length != 0:
            raise ValueError(f"{name} has {t.numel()} entries, not a multiple of {length}")
        return t.numel() // length

    def close(self):
        if getattr(self, "_ctx", None):
            lib().th_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, prec):
        _check(lib().th_set_precision(self._ctx, PREC[prec]), "th_set_precision")

    def set_variant(self, kernel, prec, variant):
        """kernel: 'fine' | 'dd' | 'coarse' | 'dd_batch' | 'resid' | 'cycle' | 'coarse_multi' | 'az' | 'coarse_refine' | 'krylov' | 'sep_sym';
        prec: 'fp64' | 'fp32'; the variant numbers are listed in include/th.h."""
        k = {"fine": 0, "dd": 1, "coarse": 6, "dd_batch": 9, "resid": 10, "cycle": 11, "coarse_multi": 12, "az": 13, "coarse_refine": 14, "krylov": 8, "sep_sym": 15}[kernel]
        _check(lib().th_set_kernel_variant(self._ctx, k, PREC[prec], int(variant)), "th_set_kernel_variant")

    def get_variant(self, kernel, prec):
        k = {"fine": 0, "dd": 1, "coarse": 6, "dd_batch": 9, "resid": 10, "cycle": 11, "coarse_multi": 12, "az": 13, "coarse_refine": 14, "krylov": 8, "sep_sym": 15}[kernel]
        v = ctypes.c_int(0)
        _check(lib().th_get_kernel_variant(self._ctx, k, PREC[prec], ctypes.byref(v)), "th_get_kernel_variant")
        return v.value

    def device_status(self):
        """Raises ThError(TH_ERR_TIMEOUT) if a bounded device wait gave up since the last check."""
        _check(lib().th_device_status(self._ctx, self._stream()), "th_device_status")

    def set_wait_limit(self, polls=-1):
        """Polls of every bounded device wait: -1 the kernels' defaults, 0 none
        (each such kernel reports a timeout and returns at once), > 0 that many."""
        _check(lib().th_set_wait_limit(self._ctx, int(polls), self._stream()), "th_set_wait_limit")

    def launch_count(self) -> int:
        v = ctypes.c_longlong(0)
        _check(lib().th_launch_count(self._ctx, ctypes.byref(v)), "th_launch_count")
        return v.value

    KERNELS = ("fine", "dd", "combine", "restrict", "prolong", "coarse_apply", "coarse_solve", "vector", "krylov")

    def profile(self, enable=True):
        """Start (clearing old records) or stop per-kernel CUDA-event timing."""
        _check(lib().th_profile(self._ctx, 1 if enable else 0), "th_profile")

    def profile_read(self):
        """{kernel class: (total ms, launches)} since profile(True)."""
        out = {}
        for i, name in enumerate(self.KERNELS):
            ms, cnt = ctypes.c_double(0), ctypes.c_longlong(0)
            _check(lib().th_profile_read(self._ctx, i, ctypes.byref(ms), ctypes.byref(cnt)), "th_profile_read")
            out[name] = (ms.value, cnt.value)
        return out

    # ------------------------------------------------------------- operators
    def apply(self, x, op="A", prec="fp64", out=None):
        length = self.Nc if op == "Aq" else self.N
        nrhs = self._vec(x, length, "x")
        y = out if out is not None else self.torch.empty_like(x)
        _check(lib().th_apply(self._ctx, OPS[op], x.data_ptr(), y.data_ptr(), nrhs, PREC[prec], self._stream()),
               "th_apply")
        return y

    def residual(self, f, u, out=None):
        nrhs = self._vec(f, self.N, "f")
        self._vec(u, self.N, "u")
        r = out if out is not None else self.torch.empty_like(f)
        _check(lib().th_residual(self._ctx, f.data_ptr(), u.data_ptr(), r.data_ptr(), nrhs, self._stream()),
               "th_residual")
        return r

    def residual_mixed(self, f, u, out=None):
        """The mixed form's outer residual f - A u, rounded to FP32 (complex64 tensor)."""
        nrhs = self._vec(f, self.N, "f")
        self._vec(u, self.N, "u")
        r = out if out is not None else self.torch.empty(f.shape, dtype=self.torch.complex64, device=self.device)
        _check(lib().th_residual_mixed(self._ctx, f.data_ptr(), u.data_ptr(), r.data_ptr(), nrhs, self._stream()),
               "th_residual_mixed")
        return r

    def smooth(self, f, u):
        """One CSDDSmoother step, in place on u."""
        nrhs = self._vec(f, self.N, "f")
        self._vec(u, self.N, "u")
        _check(lib().th_smooth(self._ctx, f.data_ptr(), u.data_ptr(), nrhs, self._stream()), "th_smooth")
        return u

    def restrict(self, r, out=None):
        nrhs = self._vec(r, self.N, "r")
        rc = out if out is not None else self.torch.empty(r.shape[:-1] + (self.Nc,), dtype=r.dtype,
                                                           device=self.device)
        _check(lib().th_restrict(self._ctx, r.data_ptr(), rc.data_ptr(), nrhs, self._stream()), "th_restrict")
        return rc

    def prolong(self, uc, u, omega=1.0):
        """u += omega * I_P uc, in place on u."""
        nrhs = self._vec(uc, self.Nc, "uc")
        self._vec(u, self.N, "u")
        _check(lib().th_prolong(self._ctx, uc.data_ptr(), u.data_ptr(), float(omega), nrhs, self._stream()),
               "th_prolong")
        return u

    def coarse_solve(self, rc, out=None):
        nrhs = self._vec(rc, self.Nc, "rc")
        uc = out if out is not None else self.torch.empty_like(rc)
        _check(lib().th_coarse_solve(self._ctx, rc.data_ptr(), uc.data_ptr(), nrhs, self._stream()),
               "th_coarse_solve")
        return uc

    def cycle(self, f, u):
        """One TwoGridStep(u, f), in place on u."""
        nrhs = self._vec(f, self.N, "f")
        self._vec(u, self.N, "u")
        _check(lib().th_cycle(self._ctx, f.data_ptr(), u.data_ptr(), nrhs, self._stream()), "th_cycle")
        return u

    def cycle_graph(self, f, u):
        """One TwoGridStep(u, f), in place on u, replayed from a captured CUDA graph."""
        nrhs = self._vec(f, self.N, "f")
        self._vec(u, self.N, "u")
        _check(lib().th_cycle_graph(self._ctx, f.data_ptr(), u.data_ptr(), nrhs, self._stream()),
               "th_cycle_graph")
        return u

    # ------------------------------------------------------- learned coarse corrector
    def unet_init(self, params, levels=4, base=16, batch_max=8):
        """params: FP32 array in the library's parameter order (th_unet_param_count entries)."""
        p = np.ascontiguousarray(params, dtype=np.float32)
        self.unet_levels = int(levels)
        _check(lib().th_unet_init(self._ctx, int(levels), int(base), int(batch_max), p.ctypes.data, p.size,
                                  self._stream()), "th_unet_init")
        self._unet_count = p.size
        mc = self.n * self.p // 2 + 1
        q = 1 << (int(levels) - 1)
        self.unet_mp = (mc + q - 1) // q * q

    def unet_params(self):
        out = np.zeros(self._unet_n(), dtype=np.float32)
        _check(lib().th_unet_get_params(self._ctx, out.ctypes.data, out.size, self._stream()), "th_unet_get_params")
        return out

    def unet_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().th_unet_set_params(self._ctx, p.ctypes.data, p.size, self._stream()), "th_unet_set_params")

    def unet_forward(self, x, out=None):
        """x: float32 CUDA tensor [B, mp, mp, 3] -> [B, mp, mp, 2]."""
        B = int(x.shape[0])
        if out is None:
            out = self.torch.empty((B, x.shape[1], x.shape[2], 2), dtype=self.torch.float32, device=x.device)
        _check(lib().th_unet_forward(self._ctx, x.data_ptr(), out.data_ptr(), B, self._stream()), "th_unet_forward")
        return out

    def unet_backward(self, gout):
        g = self.torch.empty(self._unet_n(), dtype=self.torch.float32, device=gout.device)
        _check(lib().th_unet_backward(self._ctx, gout.data_ptr(), g.data_ptr(), int(gout.shape[0]), self._stream()),
               "th_unet_backward")
        return g

    def unet_train_step(self, rc, uc, lr=1e-3):
        B = self._vec(rc, self.Nc, "rc")
        self._vec(uc, self.Nc, "uc")
        loss = ctypes.c_double(0)
        _check(lib().th_unet_train_step(self._ctx, rc.data_ptr(), uc.data_ptr(), B, float(lr), ctypes.byref(loss),
                                        self._stream()), "th_unet_train_step")
        return loss.value

    def unet_correct(self, rc, out=None):
        nrhs = self._vec(rc, self.Nc, "rc")
        uc = out if out is not None else self.torch.empty_like(rc)
        _check(lib().th_unet_correct(self._ctx, rc.data_ptr(), uc.data_ptr(), nrhs, self._stream()), "th_unet_correct")
        return uc

    def set_coarse(self, mode="direct", plain_iters=0):
        m = {"direct": 0, "learned": 1, "none": 2}[mode]
        _check(lib().th_set_coarse(self._ctx, m, int(plain_iters)), "th_set_coarse")

    def _unet_n(self):
        return self._unet_count

    def set_graphs(self, enable=True):
        _check(lib().th_set_graphs(self._ctx, 1 if enable else 0), "th_set_graphs")

    def solve(self, f, u=None, check=True):
        """FGMRES with the two-grid preconditioner; returns (u, info dict)."""
        nrhs = self._vec(f, self.N, "f")
        if u is None:
            u = self.torch.zeros_like(f)
        info = SolveInfo()
        st = lib().th_solve(self._ctx, f.data_ptr(), u.data_ptr(), nrhs, ctypes.byref(info), self._stream())
        if check and st not in (0,):
            raise ThError(st, "th_solve")
        return u, _info(info, nrhs, st)

    # host-buffer variants (copies inside the call)
    def cycle_host(self, f, u):
        f = np.ascontiguousarray(f, dtype=np.complex128)
        assert u.dtype == np.complex128 and u.flags.c_contiguous
        nrhs = f.size // self.N
        _check(lib().th_cycle_host(self._ctx, f.ctypes.data, u.ctypes.data, nrhs, self._stream()), "th_cycle_host")
        return u

    def solve_host(self, f, u=None):
        f = np.ascontiguousarray(f, dtype=np.complex128)
        nrhs = f.size // self.N
        if u is None:
            u = np.zeros_like(f)
        info = SolveInfo()
        st = lib().th_solve_host(self._ctx, f.ctypes.data, u.ctypes.data, nrhs, ctypes.byref(info), self._stream())
        if st not in (0, 4):
            raise ThError(st, "th_solve_host")
        return u, _info(info, nrhs, st)


def _info(info, nrhs, st):
    return dict(iters=info.iters, converged=info.converged, relres_max=info.relres_max,
                ms_total=info.ms_total, iters_per_rhs=list(info.iters_per_rhs[:min(nrhs, 64)]),
                fallbacks=info.fallbacks, status=st)
