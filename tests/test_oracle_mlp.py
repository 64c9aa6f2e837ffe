"""Pins for the oracle's surrogate network: the forward pass against torch's
own Linear + SiLU layers (CPU, float64), the backward pass against finite
differences of the forward pass."""
import numpy as np
import pytest

import oracle


def _params(seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(size=oracle.mlp_nparams()) * 0.3


def test_nparams():
    assert oracle.mlp_nparams() == 64 * 2 + 64 + 2 * (64 * 64 + 64) + 64 + 1 == 8577


def test_forward_against_torch():
    torch = pytest.importorskip("torch")
    P = _params(1)
    feat = np.random.default_rng(2).uniform(-1, 1, size=(50, 2))
    W1 = torch.tensor(P[:128].reshape(64, 2)); b1 = torch.tensor(P[128:192])
    W2 = torch.tensor(P[192:4288].reshape(64, 64)); b2 = torch.tensor(P[4288:4352])
    W3 = torch.tensor(P[4352:8448].reshape(64, 64)); b3 = torch.tensor(P[8448:8512])
    W4 = torch.tensor(P[8512:8576].reshape(1, 64)); b4 = torch.tensor(P[8576:8577])
    x = torch.tensor(feat)
    silu = torch.nn.functional.silu
    lin = torch.nn.functional.linear
    y = lin(silu(lin(silu(lin(silu(lin(x, W1, b1)), W2, b2)), W3, b3)), W4, b4).squeeze(1).numpy()
    assert np.allclose(oracle.mlp_forward(P, feat), y, rtol=1e-13, atol=1e-13)


def test_gradient_against_finite_differences():
    P = _params(3)
    rng = np.random.default_rng(4)
    feat = rng.uniform(-1, 1, size=(16, 2))
    t = rng.normal(size=16)
    loss, g = oracle.mlp_loss_grad(P, feat, t)
    y = oracle.mlp_forward(P, feat)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-14)
    idx = np.concatenate([rng.choice(8577, 60, replace=False), [0, 127, 128, 191, 4288, 8511, 8576]])
    for i in idx:
        h = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (np.mean((oracle.mlp_forward(Pp, feat) - t) ** 2) - np.mean((oracle.mlp_forward(Pm, feat) - t) ** 2)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_features_and_output_map():
    f = oracle.mlp_features(10.0, 0.5)
    assert f[0] == pytest.approx(1 / 3) and f[1] == 0.0
    assert oracle.mlp_features(1e-3, 1e-12)[1] == -1.0        # logit clamped at -16
    d, om = oracle.mlp_delta(1.0, 0.5)                        # zeta = 0: y = 1, delta = 3/5
    assert d == pytest.approx(0.6) and om == pytest.approx(0.4)


def _torch_bf16_network():
    """The network with bfloat16 storage written with torch: activations
    rounded in the forward pass (gradient passed straight through), the
    gradient at each pre-activation rounded in the backward pass."""
    torch = pytest.importorskip("torch")

    def q(t):
        return t.float().bfloat16().double()

    class RoundValue(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x):
            return q(x)

        @staticmethod
        def backward(ctx, g):
            return g

    class RoundGrad(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x):
            return x.clone()

        @staticmethod
        def backward(ctx, g):
            return q(g)

    def run(P, feat, t):
        Pt = torch.tensor(P, requires_grad=True)
        W1, b1 = Pt[:128].reshape(64, 2), Pt[128:192]
        W2, b2 = Pt[192:4288].reshape(64, 64), Pt[4288:4352]
        W3, b3 = Pt[4352:8448].reshape(64, 64), Pt[8448:8512]
        W4, b4 = Pt[8512:8576].reshape(1, 64), Pt[8576:8577]
        lin, silu = torch.nn.functional.linear, torch.nn.functional.silu
        h = torch.tensor(feat)
        for W, b in ((W1, b1), (W2, b2), (W3, b3)):
            h = RoundValue.apply(silu(RoundGrad.apply(lin(h, W, b))))
        y = lin(h, W4, b4).squeeze(1)
        loss = torch.mean((y - torch.tensor(t)) ** 2)
        loss.backward()
        return y.detach().numpy(), float(loss), Pt.grad.numpy()
    return run


def test_bf16_storage_network_against_torch():
    """The oracle's network with bfloat16 storage of the activations and of
    the back-propagated deltas (the rounding a kernel that stores them in
    that format applies) against torch autograd with the same rounding."""
    run = _torch_bf16_network()
    P = _params(5)
    rng = np.random.default_rng(6)
    feat = rng.uniform(-1, 1, size=(40, 2))
    t = rng.normal(size=40)
    y_t, loss_t, g_t = run(P, feat, t)
    y = oracle.mlp_forward(P, feat, bf16_storage=True)
    loss, g = oracle.mlp_loss_grad(P, feat, t, bf16_storage=True)
    assert np.allclose(y, y_t, rtol=1e-12, atol=1e-12)
    assert loss == pytest.approx(loss_t, rel=1e-12)
    assert np.allclose(g, g_t, rtol=1e-9, atol=1e-12)
    # the rounding is applied (and small): the exact network differs by it
    _, g0 = oracle.mlp_loss_grad(P, feat, t)
    d = np.linalg.norm(g - g0) / np.linalg.norm(g0)
    assert 1e-5 < d < 2e-2, d
