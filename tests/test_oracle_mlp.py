"""Pins of the FP64 surrogate-network reference: its gradient against central
finite differences of its own loss and against torch autograd (float64, a
library routine); its reference function K_ref against the closed forms it
is built to reproduce (w(iy) = erfcx(y), the Gaussian limit, the Lorentz
wing)."""
import math

import numpy as np
import pytest

from oracle import mlp

scipy_special = pytest.importorskip("scipy.special")


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    x = np.sinh(rng.uniform(0, math.asinh(10.0), n))
    y = 10 ** rng.uniform(-4, 1, n)
    keep = x * x + y * y < 100
    x, y = x[keep], y[keep]
    F = mlp.features(x, y)
    t = np.log(scipy_special.wofz(x + 1j * y).real / mlp.k_ref(x, y))
    return F, t


def test_gradient_matches_finite_differences():
    p = mlp.init_params(1)
    F, t = _batch(64, 2)
    _, g = mlp.loss_and_grad(p, F, t)
    rng = np.random.default_rng(3)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        h = 1e-6 * max(1.0, abs(p[i]))
        e[i] = h
        lp, _ = mlp.loss_and_grad(p + e, F, t)
        lm, _ = mlp.loss_and_grad(p - e, F, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-10, (i, fd, g[i])


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    p = mlp.init_params(4)
    F, t = _batch(100, 5)
    loss, g = mlp.loss_and_grad(p, F, t)
    P = {k: torch.tensor(v, requires_grad=True) for k, v in mlp.unpack(p).items()}
    Ft, tt = torch.tensor(F), torch.tensor(t)
    silu = torch.nn.functional.silu
    a = silu(Ft @ P["W1"] + P["b1"])
    a = silu(a @ P["W2"] + P["b2"])
    a = silu(a @ P["W3"] + P["b3"])
    out = a @ P["W4"] + P["b4"][0]
    L = torch.mean((out - tt) ** 2)
    L.backward()
    gt = mlp.pack({k: v.grad.numpy() for k, v in P.items()})
    assert abs(L.item() - loss) <= 1e-12 * loss
    np.testing.assert_allclose(g, gt, rtol=1e-10, atol=1e-14)


def test_reference_function_limits():
    y = np.array([1e-4, 0.1, 1.0, 5.0, 9.9])
    np.testing.assert_allclose(mlp.k_ref(np.zeros(5), y), scipy_special.erfcx(y), rtol=1e-15)
    x = np.array([0.3, 1.0, 3.0])
    np.testing.assert_allclose(mlp.k_ref(x, np.full(3, 1e-12)), np.exp(-x * x), rtol=1e-9)
    xl = np.array([50.0, 300.0])
    lor = 1.0 / (math.sqrt(math.pi) * (xl * xl + 1.0))
    np.testing.assert_allclose(mlp.k_ref(xl, np.ones(2)), lor, rtol=1e-15)
    # the residual the network learns is small over the core region
    F, t = _batch(4000, 6)
    assert np.max(np.abs(t)) < 0.5


def test_features_span_the_core_region():
    F = mlp.features(np.array([0.0, 10.0, -10.0]), np.array([1e-4, 10.0, 1.0]))
    np.testing.assert_allclose(F[:, 0], [-1.0, 1.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(F[:2, 1], [-1.0, 1.0], atol=1e-15)
