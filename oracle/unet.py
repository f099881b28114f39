"""Oracle: the learned coarse corrector, forward and backward (plain FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

The corrector has no counterpart in the paper: it stands in for the coarse
solve "u_c = A_c^{-1} r_c" of Algorithm 1 with a small convolutional U-Net on
the coarse node grid,
    u_c ~= s * UNet([Re r_c / s, Im r_c / s, eta]),   s = RMS(r_c),
with eta = k h_c averaged from the coarse cells to the nodes.  It is trained
on pairs (r_c, A_q^{-1} r_c) with the relative squared error
    loss = mean_b ||out_b - t_b||^2 / ||t_b||^2,   t_b = u_b / s_b,
over the unpadded nodes, and Adam (Kingma and Ba, 2015).

Architecture (the GPU kernels implement the same one), with L levels and C_l
= base * 2^l channels, node grid zero-padded to a multiple of 2^(L-1):
    encoder level l < L-1:  a = silu(conv3(a)) twice -> skip_l; a = avgpool2(a)
    bottom level L-1:       a = silu(conv3(a)) twice
    decoder level l:        a = [skip_l, up2(a)] (channels concatenated, skip
                            first); a = silu(conv3(a)) twice
    head:                   out = conv1(a)  (2 channels: Re, Im)
conv3: 3x3 cross-correlation with zero padding and bias; conv1: 1x1 with
bias; silu(z) = z / (1 + exp(-z)); avgpool2: mean of each 2x2 block; up2:
nearest-neighbour doubling.  Arrays are [batch, y, x, channel]; conv3 weights
are [c_out, ky, kx, c_in].

Every function is written out directly (loops over the nine taps, einsum for
the channel contractions); the backward pass is the chain rule layer by layer.
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------
# layers
# ----------------------------------------------------------------------------


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def conv3(x, w, b):
    """y[n,i,j,o] = b[o] + sum_{dy,dx,c} w[o,dy,dx,c] x[n, i+dy-1, j+dx-1, c] (zero outside)."""
    B, H, W, _ = x.shape
    xp = np.zeros((B, H + 2, W + 2, x.shape[3]))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.zeros((B, H, W, w.shape[0])) + b
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("nijc,oc->nijo", xp[:, dy:dy + H, dx:dx + W, :], w[:, dy, dx, :])
    return y


def conv3_backward(x, w, gy):
    """(dx, dw, db) of conv3 for the output gradient gy."""
    B, H, W, _ = x.shape
    xp = np.zeros((B, H + 2, W + 2, x.shape[3]))
    xp[:, 1:-1, 1:-1, :] = x
    gxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            dw[:, dy, dx, :] = np.einsum("nijo,nijc->oc", gy, xp[:, dy:dy + H, dx:dx + W, :])
            gxp[:, dy:dy + H, dx:dx + W, :] += np.einsum("nijo,oc->nijc", gy, w[:, dy, dx, :])
    return gxp[:, 1:-1, 1:-1, :], dw, gy.sum(axis=(0, 1, 2))


def conv1(x, w, b):
    """y[n,i,j,o] = b[o] + sum_c w[o,c] x[n,i,j,c]."""
    return np.einsum("nijc,oc->nijo", x, w) + b


def conv1_backward(x, w, gy):
    return np.einsum("nijo,oc->nijc", gy, w), np.einsum("nijo,nijc->oc", gy, x), gy.sum(axis=(0, 1, 2))


def avgpool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(gy):
    B, H, W, C = gy.shape
    return gy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


# ----------------------------------------------------------------------------
# network
# ----------------------------------------------------------------------------


def channels(levels: int, base: int):
    return [base * (1 << l) for l in range(levels)]


def param_shapes(levels: int, base: int, cin: int = 3, cout: int = 2):
    """Ordered (name, shape) list; the GPU library packs its parameters in this order."""
    C = channels(levels, base)
    out = []
    prev = cin
    for l in range(levels):
        out += [(f"e{l}a.w", (C[l], 3, 3, prev)), (f"e{l}a.b", (C[l],)),
                (f"e{l}b.w", (C[l], 3, 3, C[l])), (f"e{l}b.b", (C[l],))]
        prev = C[l]
    for l in range(levels - 2, -1, -1):
        out += [(f"d{l}a.w", (C[l], 3, 3, C[l] + C[l + 1])), (f"d{l}a.b", (C[l],)),
                (f"d{l}b.w", (C[l], 3, 3, C[l])), (f"d{l}b.b", (C[l],))]
    out += [("head.w", (cout, C[0])), ("head.b", (cout,))]
    return out


def forward(params, x, levels: int):
    """Network output and the cache the backward pass needs."""
    cache = {}
    skips = []
    a = x
    for l in range(levels):
        for s in "ab":
            cache[f"e{l}{s}.in"] = a
            z = conv3(a, params[f"e{l}{s}.w"], params[f"e{l}{s}.b"])
            cache[f"e{l}{s}.z"] = z
            a = silu(z)
        if l < levels - 1:
            skips.append(a)
            a = avgpool2(a)
    for l in range(levels - 2, -1, -1):
        a = np.concatenate([skips[l], up2(a)], axis=3)
        for s in "ab":
            cache[f"d{l}{s}.in"] = a
            z = conv3(a, params[f"d{l}{s}.w"], params[f"d{l}{s}.b"])
            cache[f"d{l}{s}.z"] = z
            a = silu(z)
    cache["head.in"] = a
    return conv1(a, params["head.w"], params["head.b"]), cache


def backward(params, cache, gout, levels: int):
    """Gradients of every parameter and of the input, for the output gradient gout.

    The decoder is walked from the head down (level 0 first, which was computed
    last), then the bottom level, then the encoder from the bottom up; the skip
    gradients are added to the encoder outputs they came from.
    """
    C = channels(levels, params["e0a.w"].shape[0])
    grads = {}
    g, grads["head.w"], grads["head.b"] = conv1_backward(cache["head.in"], params["head.w"], gout)
    gskip = [None] * levels
    # decoder: level 0 .. L-2 (reverse of the forward order L-2 .. 0)
    for l in range(0, levels - 1):
        for s in "ba":
            gz = g * dsilu(cache[f"d{l}{s}.z"])
            g, grads[f"d{l}{s}.w"], grads[f"d{l}{s}.b"] = conv3_backward(cache[f"d{l}{s}.in"],
                                                                        params[f"d{l}{s}.w"], gz)
        gskip[l] = g[..., :C[l]]
        g = up2_backward(g[..., C[l]:])   # gradient of the output of level l + 1
    # bottom and encoder: level L-1 .. 0
    for l in range(levels - 1, -1, -1):
        if l < levels - 1:
            g = avgpool2_backward(g) + gskip[l]
        for s in "ba":
            gz = g * dsilu(cache[f"e{l}{s}.z"])
            g, grads[f"e{l}{s}.w"], grads[f"e{l}{s}.b"] = conv3_backward(cache[f"e{l}{s}.in"],
                                                                        params[f"e{l}{s}.w"], gz)
    grads["input"] = g
    return grads


# ----------------------------------------------------------------------------
# inputs, loss, optimiser
# ----------------------------------------------------------------------------


def padded_size(m: int, levels: int) -> int:
    q = 1 << (levels - 1)
    return (m + q - 1) // q * q


def node_eta(k_coarse_cell: np.ndarray, hc: float) -> np.ndarray:
    """eta = k h_c at the coarse nodes: mean over the (up to four) adjacent coarse cells."""
    nc = k_coarse_cell.shape[0]
    m = nc + 1
    acc = np.zeros((m, m))
    cnt = np.zeros((m, m))
    for dy in (0, 1):
        for dx in (0, 1):
            acc[dy:dy + nc, dx:dx + nc] += k_coarse_cell * hc
            cnt[dy:dy + nc, dx:dx + nc] += 1.0
    return acc / cnt


def make_input(rc: np.ndarray, eta: np.ndarray, levels: int):
    """Padded network input [B, mp, mp, 3] and the scale s_b for residuals rc [B, m*m]."""
    B = rc.shape[0]
    m = eta.shape[0]
    mp = padded_size(m, levels)
    s = np.sqrt(np.mean(np.abs(rc) ** 2, axis=1))
    s = np.where(s > 0, s, 1.0)
    x = np.zeros((B, mp, mp, 3))
    r = (rc / s[:, None]).reshape(B, m, m)
    x[:, :m, :m, 0] = r.real
    x[:, :m, :m, 1] = r.imag
    x[:, :m, :m, 2] = eta
    return x, s


def loss_and_grad(out: np.ndarray, uc: np.ndarray, s: np.ndarray, m: int):
    """Relative squared error over the unpadded nodes and its gradient wrt out."""
    B = out.shape[0]
    t = (uc / s[:, None]).reshape(B, m, m)
    d = np.zeros_like(out)
    loss = 0.0
    for b in range(B):
        dr = out[b, :m, :m, 0] - t[b].real
        di = out[b, :m, :m, 1] - t[b].imag
        tn = np.sum(np.abs(t[b]) ** 2)
        loss += (np.sum(dr * dr) + np.sum(di * di)) / tn
        d[b, :m, :m, 0] = 2.0 * dr / tn / B
        d[b, :m, :m, 1] = 2.0 * di / tn / B
    return loss / B, d


def correct(params, rc: np.ndarray, eta: np.ndarray, levels: int) -> np.ndarray:
    """u_c = s UNet(rc / s) for residuals rc [B, m*m] (complex)."""
    x, s = make_input(rc, eta, levels)
    out, _ = forward(params, x, levels)
    m = eta.shape[0]
    u = out[:, :m, :m, 0] + 1j * out[:, :m, :m, 1]
    return u.reshape(rc.shape[0], m * m) * s[:, None]


class Adam:
    """theta -= lr mhat / (sqrt(vhat) + eps), with the bias-corrected moments."""

    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = {k: np.zeros_like(v) for k, v in params.items()}
        self.v = {k: np.zeros_like(v) for k, v in params.items()}
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        for k in params:
            g = grads[k]
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * g
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * g * g
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            params[k] = params[k] - self.lr * mh / (np.sqrt(vh) + self.eps)
