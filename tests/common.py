"""Shared helpers for the tests: problem builders for the oracle and the library."""
import numpy as np

import synth

SIDE_TO_ORACLE = {"xlo": (1, 0), "xhi": (1, 1), "ylo": (0, 0), "yhi": (0, 1)}


def oracle_bc(bc):
    """Binding boundary spec -> oracle spec ({(axis, end): kind})."""
    if isinstance(bc, str):
        return bc
    return {SIDE_TO_ORACLE[s]: v for s, v in bc.items()}


def small_case(n=6, p=4, W=1.5, seed=3, layer=6.0):
    k = synth.random_wavenumber(n, 2, W, seed=seed)
    eps = synth.absorbing_layer(n, 2, p, k, layer)
    return k, eps


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def ensure_built():
    import __graft_entry__
    __graft_entry__.build()
