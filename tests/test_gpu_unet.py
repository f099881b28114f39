"""Learned coarse corrector on the GPU against the FP64 oracle (oracle/unet.py).

Tolerances: the network runs with BF16 weights and activations (unit roundoff
2^-9) and FP32 accumulation, through ~15 layers; the oracle gets the same
BF16-rounded weights, so what remains is the rounding of the activations:
outputs within 3e-2 (max-norm relative), parameter gradients within 5e-2
(2-norm relative per tensor).  Training, the solve with the corrector inside
FGMRES and its fallback are checked by behaviour (loss decrease, convergence,
iterations against the smoother-only method)."""
import numpy as np
import pytest

import synth
from oracle import unet as ounet
from tests.common import ensure_built

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"
LEVELS, BASE = 4, 16


@pytest.fixture(scope="module")
def th():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_2509_17494_gb300 as th
    return th


def bf16_round(a):
    """Round FP32 values to the nearest BF16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(flat, shapes):
    out, off = {}, 0
    for name, shape in shapes:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    return out


@pytest.fixture(scope="module")
def case(th):
    w = synth.workload("square10_q4_n25")
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5, l_dd=2, prec="bf16",
                         extra_prec=("fp64",), nrhs_max=8, restart=40, device=DEV)
    shapes = th.unet_param_shapes(LEVELS, BASE)
    params0 = synth.he_normal(shapes, 77)
    S.unet_init(params0, levels=LEVELS, base=BASE, batch_max=8)
    return S, w, shapes, params0


def test_param_order_matches_oracle(th):
    assert th.unet_param_shapes(3, 16) == ounet.param_shapes(3, 16)
    assert th.unet_param_count(4, 16) == sum(int(np.prod(s)) for _, s in ounet.param_shapes(4, 16))


def test_forward_matches_oracle(case):
    S, w, shapes, params0 = case
    mp = S.unet_mp
    x = synth.rng(3).standard_normal((2, mp, mp, 3)).astype(np.float32)
    got = S.unet_forward(torch.from_numpy(x).to(DEV)).cpu().numpy()
    P = unflatten(bf16_round(params0), shapes)
    for k in P:
        if k.endswith(".b") or k.startswith("head"):
            P[k] = unflatten(params0, shapes)[k]   # biases and the head stay FP32 on the GPU
    want, _ = ounet.forward(P, bf16_round(x), LEVELS)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 3e-2, err
    # deterministic
    again = S.unet_forward(torch.from_numpy(x).to(DEV)).cpu().numpy()
    assert np.array_equal(got, again)


def test_backward_matches_oracle(case):
    S, w, shapes, params0 = case
    mp = S.unet_mp
    r = synth.rng(4)
    x = r.standard_normal((2, mp, mp, 3)).astype(np.float32)
    gout = r.standard_normal((2, mp, mp, 2)).astype(np.float32)
    S.unet_forward(torch.from_numpy(x).to(DEV))
    got = S.unet_backward(torch.from_numpy(gout).to(DEV)).cpu().numpy()
    P = unflatten(bf16_round(params0), shapes)
    for k in P:
        if k.endswith(".b") or k.startswith("head"):
            P[k] = unflatten(params0, shapes)[k]
    _, cache = ounet.forward(P, bf16_round(x), LEVELS)
    want = ounet.backward(P, cache, gout.astype(np.float64), LEVELS)
    G = unflatten(got, shapes)
    for name, _ in shapes:
        e = np.linalg.norm(G[name] - want[name]) / max(np.linalg.norm(want[name]), 1e-30)
        assert e < 5e-2, (name, e)


def _pairs(S, w, count, seed):
    """Coarse residuals (half restricted fine residuals after one smoothing, half
    smooth coarse noise) and their direct coarse solutions (FP64)."""
    m = S.n * S.p // 2 + 1
    half = count // 2
    f = torch.from_numpy(synth.random_complex((half, S.N), seed)).to(DEV)
    S.set_precision("fp64")
    u = torch.zeros_like(f)
    S.smooth(f, u)
    rc1 = S.restrict(S.residual(f, u))
    rc2 = torch.from_numpy(synth.smooth_coarse_noise(m, count - half, seed + 1)).to(DEV)
    rc = torch.cat([rc1, rc2]).contiguous()
    uc = torch.cat([S.coarse_solve(rc[i:i + 8].contiguous()) for i in range(0, count, 8)]).contiguous()
    S.set_precision("bf16")
    return rc, uc


def test_loss_matches_oracle_and_training_reduces_it(case):
    S, w, shapes, params0 = case
    S.unet_set_params(params0)
    rc, uc = _pairs(S, w, 8, 10)
    # the loss reported by the first step is the loss of the initial parameters
    m = S.n * S.p // 2 + 1
    eta = ounet.node_eta(np.repeat(np.repeat(w["k"], 2, 0), 2, 1), 1.0 / (m - 1))
    P = unflatten(params0, shapes)
    x, s = ounet.make_input(rc.cpu().numpy(), eta, LEVELS)
    out, _ = ounet.forward(P, x, LEVELS)
    want, _ = ounet.loss_and_grad(out, uc.cpu().numpy(), s, m)
    got = S.unet_train_step(rc, uc, lr=1e-3)
    assert abs(got - want) / want < 5e-2, (got, want)
    # a short training run on fresh pairs
    losses = []
    for it in range(150):
        if it % 10 == 0:
            rc, uc = _pairs(S, w, 8, 100 + it)
        losses.append(S.unet_train_step(rc, uc, lr=2e-3))
    assert np.mean(losses[-10:]) < 0.7 * np.mean(losses[:10]), (losses[:10], losses[-10:])
    torch.cuda.synchronize()
    S.device_status()


def test_learned_corrector_in_fgmres(case, th):
    """After the training above: the correction equals the oracle's for the
    trained parameters, FGMRES converges with the corrector (falling back to the
    direct solve if it would exceed 1.5 x the plain count), and it needs fewer
    iterations than the smoother alone."""
    S, w, shapes, _ = case
    trained = S.unet_params()
    m = S.n * S.p // 2 + 1
    rc, _ = _pairs(S, w, 4, 500)
    got = S.unet_correct(rc).cpu().numpy()
    P = unflatten(bf16_round(trained), shapes)
    for k in P:
        if k.endswith(".b") or k.startswith("head"):
            P[k] = unflatten(trained, shapes)[k]
    eta = ounet.node_eta(np.repeat(np.repeat(w["k"], 2, 0), 2, 1), 1.0 / (m - 1))
    want = ounet.correct(P, rc.cpu().numpy(), eta, LEVELS)
    assert np.abs(got - want).max() / np.abs(want).max() < 5e-2

    f = torch.from_numpy(w["f"]).to(DEV)
    S.set_coarse("direct")
    _, plain = S.solve(f)
    S.set_coarse("none")
    _, none = S.solve(f, check=False)
    S.set_coarse("learned", plain_iters=plain["iters"])
    u, learned = S.solve(f, check=False)
    S.set_coarse("direct")
    assert learned["converged"] == 1 and learned["relres_max"] <= 1e-8 * 1.0001
    assert learned["iters"] <= none["iters"] or none["converged"] == 0
    if learned["fallbacks"] == 0:
        assert learned["iters"] < int(np.ceil(1.5 * plain["iters"])) + 1
    # without a fallback count the learned solve may not stop early
    S.set_coarse("learned", plain_iters=0)
    _, free = S.solve(f, check=False)
    S.set_coarse("direct")
    assert free["fallbacks"] == 0


def test_32_channel_network_matches_oracle(th):
    """The configuration-4 width: 4 levels of 32 base channels.  The decoder's
    widest concatenation (128 + 256 = 384 channels) makes its input gradient an
    MMA of N = 384 > 256, run as two launches over output-channel ranges."""
    w = synth.workload("square10_q4_n25")
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5, l_dd=2, prec="bf16",
                         extra_prec=("fp64",), nrhs_max=2, device=DEV)
    shapes = th.unet_param_shapes(4, 32)
    assert shapes == ounet.param_shapes(4, 32)
    params0 = synth.he_normal(shapes, 78)
    S.unet_init(params0, levels=4, base=32, batch_max=2)
    mp = S.unet_mp
    r = synth.rng(5)
    x = r.standard_normal((2, mp, mp, 3)).astype(np.float32)
    gout = r.standard_normal((2, mp, mp, 2)).astype(np.float32)
    got = S.unet_forward(torch.from_numpy(x).to(DEV)).cpu().numpy()
    grads = S.unet_backward(torch.from_numpy(gout).to(DEV)).cpu().numpy()
    S.device_status()
    P = unflatten(bf16_round(params0), shapes)
    for k in P:
        if k.endswith(".b") or k.startswith("head"):
            P[k] = unflatten(params0, shapes)[k]
    want, cache = ounet.forward(P, bf16_round(x), 4)
    assert np.abs(got - want).max() / np.abs(want).max() < 3e-2
    gw = ounet.backward(P, cache, gout.astype(np.float64), 4)
    G = unflatten(grads, shapes)
    for name, _ in shapes:
        e = np.linalg.norm(G[name] - gw[name]) / max(np.linalg.norm(gw[name]), 1e-30)
        assert e < 5e-2, (name, e)
    S.close()
