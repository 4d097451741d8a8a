"""FP64 reference of the Voigt-function surrogate network.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The CUDA library trains
and evaluates its own BF16 tensor-core version; this module is what its
forward pass and its loss gradients are checked against.

Network (2 -> 64 -> 64 -> 64 -> 1, SiLU): it stands in for the Voigt function
K(x, y) = Re w(x + iy) where the method uses Algorithm 916 (Sec. 2.4:
x^2 + y^2 < 100), in the form

  K(x, y) = K_ref(x, y) * exp(net(f1, f2)),
  K_ref   = e^{-x^2} erfcx(y) + (1 - e^{-x^2}) y / (sqrt(pi) (x^2 + y^2)),
  f1 = 2 asinh|x| / asinh(10) - 1,   f2 = 2 (log10 y + 4) / 5 - 1,

so the network learns the small residual ln(K / K_ref) (|.| < 0.4): K_ref is
exact at x = 0 (w(iy) = erfcx y), at y -> 0 (the Gaussian) and in the
Lorentz far wing.

Parameters, flat FP32/FP64 vector of N_PARAMS values in this order:
W1 [2][64], b1 [64], W2 [64][64], b2 [64], W3 [64][64], b3 [64], W4 [64], b4
(W[in][out]; z = a W + b).  Loss: mean squared error of the residual.
"""
import math

import numpy as np

H = 64
N_PARAMS = 2 * H + H + H * H + H + H * H + H + H + 1
X_CORE = 10.0
LOGY_MIN, LOGY_MAX = -4.0, 1.0


def features(x, y):
    x = np.abs(np.asarray(x, dtype=np.float64))
    y = np.asarray(y, dtype=np.float64)
    f1 = 2.0 * np.arcsinh(x) / math.asinh(X_CORE) - 1.0
    f2 = 2.0 * (np.log10(y) - LOGY_MIN) / (LOGY_MAX - LOGY_MIN) - 1.0
    return np.stack([f1, f2], axis=1)


def k_ref(x, y):
    from scipy.special import erfcx
    x = np.abs(np.asarray(x, dtype=np.float64))
    y = np.asarray(y, dtype=np.float64)
    e = np.exp(-x * x)
    return e * erfcx(y) + (1.0 - e) * y / (math.sqrt(math.pi) * (x * x + y * y))


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    assert p.shape == (N_PARAMS,)
    o = 0
    out = {}
    for name, shape in (("W1", (2, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                        ("W3", (H, H)), ("b3", (H,)), ("W4", (H,)), ("b4", (1,))):
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[k], dtype=np.float64).ravel()
                           for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")])


def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(p, F):
    """Residual prediction for features F (N, 2); returns (out, cache)."""
    P = unpack(p)
    z1 = F @ P["W1"] + P["b1"]
    a1 = z1 * _sig(z1)
    z2 = a1 @ P["W2"] + P["b2"]
    a2 = z2 * _sig(z2)
    z3 = a2 @ P["W3"] + P["b3"]
    a3 = z3 * _sig(z3)
    out = a3 @ P["W4"] + P["b4"][0]
    return out, (F, z1, a1, z2, a2, z3, a3)


def loss_and_grad(p, F, t):
    """Mean squared error of the residual and its gradient (flat vector)."""
    P = unpack(p)
    out, (F, z1, a1, z2, a2, z3, a3) = forward(p, F)
    n = F.shape[0]
    r = out - t
    loss = float(np.mean(r * r))
    dout = 2.0 * r / n

    def dsilu(z):
        s = _sig(z)
        return s * (1.0 + z * (1.0 - s))

    g = {"W4": a3.T @ dout, "b4": np.array([dout.sum()])}
    dz3 = np.outer(dout, P["W4"]) * dsilu(z3)
    g["W3"] = a2.T @ dz3
    g["b3"] = dz3.sum(axis=0)
    dz2 = (dz3 @ P["W3"].T) * dsilu(z2)
    g["W2"] = a1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"].T) * dsilu(z1)
    g["W1"] = F.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def predict_k(p, x, y):
    out, _ = forward(p, features(x, y))
    return k_ref(x, y) * np.exp(out)


def init_params(seed):
    """Seeded He-style initialisation (used only by tests)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, math.sqrt(2.0 / 2), (2, H)), "b1": np.zeros(H),
         "W2": rng.normal(0, math.sqrt(2.0 / H), (H, H)), "b2": np.zeros(H),
         "W3": rng.normal(0, math.sqrt(2.0 / H), (H, H)), "b3": np.zeros(H),
         "W4": rng.normal(0, math.sqrt(1.0 / H), H), "b4": np.zeros(1)}
    return pack(d)
