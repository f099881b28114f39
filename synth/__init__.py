"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module holds problem DATA only (wavenumber and damping fields per cell,
right-hand sides, random vectors).  It contains none of the solver's
arithmetic: no basis functions, no element matrices, no stencils.  Both the
oracle and the GPU library receive the arrays produced here unchanged.

Problem statement (Section 2, Eq. Helmholtz_eq): -Lap u - (k^2 + i eps) u = f on
the unit square (or cube), with k and eps constant per cell of the underlying
uniform mesh of n cells per direction.

Workload recipe (all seeds fixed):
  * constant k = 2*pi*W for a domain of W wavelengths;
  * random velocity field: white noise from numpy's PCG64(seed) on the cell
    centre grid, Gaussian-filtered in Fourier space with correlation length
    ell = 1/8, normalised to zero mean and max |g| = 1; c = 1 + 0.3 g and
    k = k0 / c (so +/-30% velocity contrast);
  * absorbing layer (Section 7): eps rises with a sin^2 profile from 0 at the
    inner edge of a layer of `width_dofs` dof spacings to 2 k^2 / pi at the
    outer boundary, evaluated at cell centres, maximum over the sides;
  * sources are load vectors (dual vectors) given directly on the dof grid: a
    discrete Gaussian of one dof spacing in index space, normalised to unit sum.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2509


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def constant_wavenumber(n: int, dim: int, wavelengths: float) -> np.ndarray:
    """k per cell for a domain of `wavelengths` wavelengths (unit length)."""
    return np.full((n,) * dim, 2.0 * np.pi * wavelengths)


def random_velocity(n: int, dim: int, seed: int, ell: float = 1.0 / 8.0,
                    contrast: float = 0.3) -> np.ndarray:
    """Smooth Gaussian random velocity c(x) per cell, mean 1, max |c-1| = contrast."""
    w = rng(seed).standard_normal((n,) * dim)
    kap = 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n)
    grids = np.meshgrid(*([kap] * dim), indexing="ij")
    k2 = sum(g * g for g in grids)
    filt = np.exp(-0.5 * k2 * ell * ell)
    g = np.real(np.fft.ifftn(np.fft.fftn(w) * filt))
    g -= g.mean()
    g /= np.abs(g).max()
    return 1.0 + contrast * g


def random_wavenumber(n: int, dim: int, wavelengths: float, seed: int) -> np.ndarray:
    """k = k0 / c with k0 = 2 pi * wavelengths and c a seeded random velocity."""
    return 2.0 * np.pi * wavelengths / random_velocity(n, dim, seed)


def absorbing_layer(n: int, dim: int, p: int, k_cell: np.ndarray,
                    width_dofs: float = 10.0) -> np.ndarray:
    """eps per cell: sin^2 ramp from 0 to 2 k^2/pi over `width_dofs` dof spacings.

    Depth d is measured inward from the inner edge of the layer; the profile is
    (2 k^2/pi) sin^2(pi d / (2 w)) with w = width_dofs * h / p, evaluated at
    cell centres and maximised over all sides of the box.
    """
    h = 1.0 / n
    w = width_dofs * h / p
    centres = (np.arange(n) + 0.5) * h
    dist = np.minimum(centres, 1.0 - centres)          # distance to nearest side, per axis
    depth1 = np.clip(w - dist, 0.0, None)               # depth into the layer, per axis
    grids = np.meshgrid(*([depth1] * dim), indexing="ij")
    depth = np.maximum.reduce(grids)
    prof = np.sin(0.5 * np.pi * depth / w) ** 2
    return (2.0 * k_cell ** 2 / np.pi) * prof


def min_points_per_wavelength(k_cell: np.ndarray, n: int, p: int) -> float:
    """Smallest dofs per wavelength over the cells: 2 pi p / (k h)."""
    return float(2.0 * np.pi * p * n / k_cell.max())


def gaussian_source(n: int, p: int, dim: int, centre_index=None,
                    sigma: float = 1.0) -> np.ndarray:
    """Load vector: discrete Gaussian on the dof grid (index units), unit sum.

    Returned as a complex array of shape (N,) in lexicographic order, x fastest.
    """
    m = n * p + 1
    if centre_index is None:
        centre_index = [0.5 * (m - 1)] * dim
    idx = np.arange(m, dtype=float)
    grids = np.meshgrid(*([idx] * dim), indexing="ij")  # grids[0] = slowest axis
    # axis order: array index 0 is the slowest (z or y), the last is x.
    r2 = sum((g - c) ** 2 for g, c in zip(grids, reversed(list(centre_index))))
    f = np.exp(-0.5 * r2 / sigma ** 2)
    f /= f.sum()
    return f.reshape(-1).astype(np.complex128)


def random_sources(n: int, p: int, dim: int, count: int, seed: int,
                   margin_dofs: int = 12) -> np.ndarray:
    """`count` Gaussian sources at seeded random dof positions away from the layer.

    Shape (count, N), complex128.
    """
    m = n * p + 1
    r = rng(seed)
    out = np.empty((count, m ** dim), dtype=np.complex128)
    for s in range(count):
        c = r.integers(margin_dofs, m - margin_dofs, size=dim).astype(float)
        out[s] = gaussian_source(n, p, dim, centre_index=list(c))
    return out


def random_complex(shape, seed: int) -> np.ndarray:
    """Standard complex normal array (independent real/imaginary parts)."""
    r = rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


# Named workloads.  Sizes follow the paper's experiments (Section 7) and the
# configurations the library is measured on.
def workload(name: str):
    """Return a dict describing one of the named synthetic workloads."""
    if name == "square10_q4_n25":       # 10 wavelengths, Q4, 25x25 cells, 101^2 dofs
        n, p, W = 25, 4, 10.0
        k = constant_wavenumber(n, 2, W)
        eps = np.zeros_like(k)
        return dict(name=name, dim=2, n=n, p=p, k=k, eps=eps, bc="robin",
                    f=gaussian_source(n, p, 2), alpha_s=0.5, l_dd=2)
    if name == "square40_q4_n100":      # 40 wavelengths, Q4, 100x100 cells, 401^2 dofs
        n, p, W = 100, 4, 40.0
        k = random_wavenumber(n, 2, W, seed=1)
        eps = absorbing_layer(n, 2, p, k, 10.0)
        return dict(name=name, dim=2, n=n, p=p, k=k, eps=eps, bc="robin",
                    f=gaussian_source(n, p, 2), alpha_s=0.5, l_dd=2)
    if name == "square80_q4_n200":      # 80 wavelengths, Q4, 200x200 cells, 801^2 dofs
        n, p, W = 200, 4, 80.0
        k = random_wavenumber(n, 2, W, seed=1)
        eps = absorbing_layer(n, 2, p, k, 10.0)
        return dict(name=name, dim=2, n=n, p=p, k=k, eps=eps, bc="robin",
                    f=random_sources(n, p, 2, 64, seed=100), alpha_s=0.5, l_dd=2)
    if name == "cube10_q2_n40":         # 3-D, 10 wavelengths, Q2, 40^3 cells, 81^3 dofs, 8 sources
        n, p, W = 40, 2, 10.0
        k = random_wavenumber(n, 3, W, seed=1)
        eps = absorbing_layer(n, 3, p, k, 10.0)
        return dict(name=name, dim=3, n=n, p=p, k=k, eps=eps, bc="robin",
                    f=random_sources(n, p, 3, 8, seed=100, margin_dofs=12), alpha_s=0.5, l_dd=2)
    if name == "cube2_q2_n8":           # small 3-D case: 2 wavelengths, Q2, 8^3 cells, 17^3 dofs
        n, p, W = 8, 2, 2.0
        k = random_wavenumber(n, 3, W, seed=3)
        eps = absorbing_layer(n, 3, p, k, 3.0)
        return dict(name=name, dim=3, n=n, p=p, k=k, eps=eps, bc="robin",
                    f=gaussian_source(n, p, 3), alpha_s=0.5, l_dd=2)
    raise KeyError(name)


def he_normal(shapes, seed: int) -> np.ndarray:
    """Initial parameters of the learned coarse corrector: for each (name, shape)
    in order, weights (names ending in ".w") drawn N(0, 2 / fan_in) with fan_in the
    product of the trailing dimensions, biases zero; flattened to one float32 array."""
    r = rng(seed)
    out = []
    for name, shape in shapes:
        n = int(np.prod(shape))
        if name.endswith(".w"):
            fan_in = int(np.prod(shape[1:]))
            out.append(r.standard_normal(n) * np.sqrt(2.0 / fan_in))
        else:
            out.append(np.zeros(n))
    return np.concatenate(out).astype(np.float32)


def smooth_coarse_noise(m: int, count: int, seed: int, passes: int = 4) -> np.ndarray:
    """Complex white noise on an m x m node grid, averaged `passes` times with its
    4 neighbours (zero outside): smooth random coarse residuals, [count, m*m]."""
    r = rng(seed)
    z = r.standard_normal((count, m, m)) + 1j * r.standard_normal((count, m, m))
    for _ in range(passes):
        zp = np.zeros((count, m + 2, m + 2), dtype=complex)
        zp[:, 1:-1, 1:-1] = z
        z = (zp[:, 1:-1, 1:-1] * 2 + zp[:, :-2, 1:-1] + zp[:, 2:, 1:-1] + zp[:, 1:-1, :-2] + zp[:, 1:-1, 2:]) / 6.0
    return z.reshape(count, m * m)

