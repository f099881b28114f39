"""Pins of the learned-corrector oracle (FP64, CPU) against facts that do not
come from the oracle itself: a library cross-correlation, finite differences,
adjoint identities and the closed form of Adam's first step."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import unet
import synth


def _params(levels, base, seed, scale=0.3):
    r = synth.rng(seed)
    return {k: scale * r.standard_normal(s) for k, s in unet.param_shapes(levels, base)}


def test_conv3_is_library_cross_correlation():
    r = synth.rng(1)
    x = r.standard_normal((2, 7, 9, 3))
    w = r.standard_normal((4, 3, 3, 3))
    b = r.standard_normal(4)
    y = unet.conv3(x, w, b)
    for n in range(2):
        for o in range(4):
            want = b[o] + sum(correlate2d(x[n, :, :, c], w[o, :, :, c], mode="same") for c in range(3))
            assert np.allclose(y[n, :, :, o], want, rtol=0, atol=1e-12)


def test_pool_and_upsample_adjoints():
    r = synth.rng(2)
    x = r.standard_normal((2, 8, 6, 3))
    y = r.standard_normal((2, 4, 3, 3))
    assert np.isclose(np.sum(unet.avgpool2(x) * y), np.sum(x * unet.avgpool2_backward(y)))
    assert np.isclose(np.sum(unet.up2(y) * x), np.sum(y * unet.up2_backward(x)))
    # averaging a doubled field returns it
    assert np.allclose(unet.avgpool2(unet.up2(y)), y)


def test_silu_derivative_finite_difference():
    z = np.linspace(-6, 6, 41)
    h = 1e-6
    fd = (unet.silu(z + h) - unet.silu(z - h)) / (2 * h)
    assert np.allclose(unet.dsilu(z), fd, atol=1e-9)


@pytest.mark.parametrize("levels,base", [(2, 2), (3, 2)])
def test_backward_matches_finite_differences(levels, base):
    """Every parameter tensor (sampled entries) and the input: d(sum out * R)/d theta."""
    params = _params(levels, base, 3)
    r = synth.rng(4)
    H = 4 * (1 << (levels - 1))
    x = r.standard_normal((2, H, H, 3))
    R = r.standard_normal((2, H, H, 2))
    out, cache = unet.forward(params, x, levels)
    grads = unet.backward(params, cache, R, levels)

    def objective(p, xx):
        return float(np.sum(unet.forward(p, xx, levels)[0] * R))

    h = 1e-6
    pick = synth.rng(5)
    for name, shape in unet.param_shapes(levels, base):
        flat = params[name].reshape(-1)
        for idx in pick.choice(flat.size, size=min(4, flat.size), replace=False):
            keep = flat[idx]
            flat[idx] = keep + h
            fp = objective(params, x)
            flat[idx] = keep - h
            fm = objective(params, x)
            flat[idx] = keep
            fd = (fp - fm) / (2 * h)
            g = grads[name].reshape(-1)[idx]
            assert abs(g - fd) <= 1e-6 * max(1.0, abs(fd)), (name, idx, g, fd)
    xf = x.reshape(-1)
    for idx in pick.choice(xf.size, size=6, replace=False):
        keep = xf[idx]
        xf[idx] = keep + h
        fp = objective(params, x)
        xf[idx] = keep - h
        fm = objective(params, x)
        xf[idx] = keep
        assert abs(grads["input"].reshape(-1)[idx] - (fp - fm) / (2 * h)) <= 1e-6 * max(1.0, abs(fp - fm) / (2 * h))


def test_loss_gradient_finite_difference():
    r = synth.rng(6)
    m, mp, B = 5, 8, 2
    out = r.standard_normal((B, mp, mp, 2))
    uc = synth.random_complex((B, m * m), 7)
    s = np.array([0.5, 2.0])
    L, d = unet.loss_and_grad(out, uc, s, m)
    # the loss is zero at the target and the padding carries no gradient
    assert np.all(d[:, m:, :, :] == 0) and np.all(d[:, :, m:, :] == 0)
    h = 1e-6
    for idx in [(0, 1, 2, 0), (1, 4, 0, 1), (1, 3, 3, 0)]:
        o2 = out.copy()
        o2[idx] += h
        lp = unet.loss_and_grad(o2, uc, s, m)[0]
        o2[idx] -= 2 * h
        lm = unet.loss_and_grad(o2, uc, s, m)[0]
        assert abs(d[idx] - (lp - lm) / (2 * h)) < 1e-7
    t = (uc / s[:, None]).reshape(B, m, m)
    exact = np.zeros_like(out)
    exact[:, :m, :m, 0] = t.real
    exact[:, :m, :m, 1] = t.imag
    assert unet.loss_and_grad(exact, uc, s, m)[0] == 0.0


def test_adam_first_step_closed_form():
    """After one step from zero moments, mhat = g and vhat = g^2: theta -= lr g / (|g| + eps)."""
    params = {"a": np.array([1.0, -2.0, 3.0])}
    g = {"a": np.array([0.5, -1e-3, 0.0])}
    opt = unet.Adam(params, lr=0.1, eps=1e-8)
    opt.step(params, g)
    want = np.array([1.0, -2.0, 3.0]) - 0.1 * g["a"] / (np.abs(g["a"]) + 1e-8)
    assert np.allclose(params["a"], want, rtol=0, atol=1e-12)


def test_inputs_and_correction_scale_invariance():
    kc = np.full((4, 4), 12.0)
    eta = unet.node_eta(kc, 0.25)
    assert eta.shape == (5, 5) and np.allclose(eta, 3.0)
    rc = synth.random_complex((2, 25), 8)
    x, s = unet.make_input(rc, eta, levels=2)
    assert x.shape == (2, 6, 6, 3)
    assert np.allclose(s, np.sqrt(np.mean(np.abs(rc) ** 2, axis=1)))
    assert np.allclose(np.mean(x[:, :5, :5, 0] ** 2 + x[:, :5, :5, 1] ** 2, axis=(1, 2)), 1.0)
    params = _params(2, 2, 9)
    u1 = unet.correct(params, rc, eta, 2)
    u2 = unet.correct(params, 7.5 * rc, eta, 2)
    assert np.allclose(u2, 7.5 * u1)
