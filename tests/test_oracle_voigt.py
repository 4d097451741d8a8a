"""Pins of the oracle's Voigt function (Sec. 2.3-2.4) against references that
do not reuse its formulas: mpmath's w(z), scipy's erfcx, numpy's
Gauss-Hermite nodes, scipy quadrature of the convolution integral."""
import math

import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")
scipy_special = pytest.importorskip("scipy.special")
scipy_integrate = pytest.importorskip("scipy.integrate")

mpmath.mp.dps = 30


def w_exact_re(x, y):
    z = mpmath.mpc(x, y)
    return float(mpmath.re(mpmath.exp(-z * z) * mpmath.erfc(-1j * z)))


def _core_points(n, seed):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        r = 10.0 * math.sqrt(rng.random())
        th = rng.random() * math.pi / 2
        x, y = r * math.cos(th), r * math.sin(th)
        if rng.random() < 0.3:
            y = 10.0 ** rng.uniform(-12, 0)
        if x * x + y * y < 100.0:
            pts.append((x, y))
    return pts


def test_k916_matches_mpmath_over_core_region():
    # Algorithm 916 (Sec. 2.4) is accurate to ~1e-15; the oracle's erfcx
    # (exp(y^2) erfc(y)) costs up to ~1e-14 near y = 10.
    worst = 0.0
    for x, y in _core_points(1500, 1):
        k = oracle.K916(x, y)
        ke = w_exact_re(x, y)
        worst = max(worst, abs(k - ke) / ke)
    assert worst < 2e-14, worst


def test_k916_lattice_corners():
    for x in (0.0, 1e-8, 0.5, 2.0, 5.0, 9.999):
        for y in (0.0, 1e-10, 1e-4, 0.3, 3.0, 9.99):
            if x * x + y * y >= 100.0:
                continue
            ke = w_exact_re(x, y)
            assert abs(oracle.K916(x, y) - ke) <= 2e-14 * ke + 1e-300


def test_k916_imaginary_axis_is_erfcx():
    # w(iy) = erfcx(y)  (closed form)
    for y in np.linspace(0.0, 9.99, 37):
        ref = scipy_special.erfcx(y)
        assert abs(oracle.K916(0.0, y) - ref) <= 2e-14 * ref


def test_k916_gaussian_limit():
    # y -> 0: H(0, u) = exp(-u^2)  (Doppler limit of the Voigt profile)
    for x in np.linspace(0.0, 9.0, 31):
        ref = math.exp(-x * x)
        assert abs(oracle.K916(x, 0.0) - ref) <= 1e-14 * ref


def test_k916_even_in_x():
    for x, y in _core_points(50, 2):
        assert oracle.K916(x, y) == oracle.K916(-x, y)


def test_gh3_is_the_three_node_hermite_rule():
    # nodes/weights from numpy (roots of H_3), not from the oracle's constants
    t, w = np.polynomial.hermite.hermgauss(3)
    rng = np.random.default_rng(3)
    for _ in range(200):
        x = rng.uniform(-1000, 1000)
        y = 10 ** rng.uniform(-6, 2)
        ref = (y / math.pi) * sum(wk / ((x - tk) ** 2 + y * y) for tk, wk in zip(t, w))
        assert abs(oracle.gh3(x, y) - ref) <= 1e-14 * ref


def test_gh1_is_lorentz_far_wing():
    t, w = np.polynomial.hermite.hermgauss(1)
    assert t[0] == 0.0 and abs(w[0] - math.sqrt(math.pi)) < 1e-15
    for x, y in [(1e3, 1.0), (3e3, 1e-3), (1e5, 50.0), (-2e4, 7.0)]:
        ref = y / (math.sqrt(math.pi) * (x * x + y * y))
        assert abs(oracle.gh1(x, y) - ref) <= 1e-15 * ref


def test_gauss_hermite_regions_within_method_error():
    # Within the method's own accuracy: GH3 <= 6e-6 on 100 <= r^2 < 1e6,
    # GH1 <= 2e-6 on r^2 >= 1e6 (relative to the exact w).
    rng = np.random.default_rng(4)
    worst3 = worst1 = 0.0
    for _ in range(300):
        r = math.sqrt(10 ** rng.uniform(2, 6))
        th = rng.random() * math.pi / 2
        x, y = r * math.cos(th), r * math.sin(th)
        if x * x + y * y < 100.0 or x * x + y * y >= 1e6:
            continue
        worst3 = max(worst3, abs(oracle.gh3(x, y) / w_exact_re(x, y) - 1))
    for _ in range(300):
        r = math.sqrt(10 ** rng.uniform(6, 10))
        th = rng.random() * math.pi / 2
        x, y = r * math.cos(th), r * math.sin(th)
        if x * x + y * y < 1e6:
            continue
        worst1 = max(worst1, abs(oracle.gh1(x, y) / w_exact_re(x, y) - 1))
    assert worst3 < 6e-6, worst3
    assert worst1 < 2e-6, worst1


def test_region_dispatch_thresholds():
    a = 0.5
    u100 = math.sqrt(100.0 - a * a)
    below = np.nextafter(u100, 0)
    above = np.nextafter(u100, 1e9)
    assert oracle.voigt_H(a, below)[1] == 0
    assert oracle.voigt_H(a, above)[1] == 1
    u1e6 = math.sqrt(1e6 - a * a)
    assert oracle.voigt_H(a, np.nextafter(u1e6, 0))[1] == 1
    assert oracle.voigt_H(a, np.nextafter(u1e6, 1e9))[1] == 2
    # the values chosen are those of the selected method
    assert oracle.voigt_H(a, below)[0] == oracle.K916(below, a)
    assert oracle.voigt_H(a, above)[0] == oracle.gh3(above, a)


def test_voigt_is_gauss_lorentz_convolution():
    # H(a,u) = (a/pi) int exp(-t^2) / ((u-t)^2 + a^2) dt by adaptive quadrature
    for a, u in [(1e-3, 0.0), (0.05, 1.2), (0.5, 3.0), (1.0, 0.0), (2.0, 6.0),
                 (3.0, 12.0), (0.2, 40.0), (7.0, 80.0), (30.0, 5.0), (0.01, 9.5)]:
        f = lambda t: math.exp(-t * t) / ((u - t) ** 2 + a * a)
        pts = sorted({-6.0, 6.0, u - a, u, u + a})
        pts = [p for p in pts if -30 < p < 30]
        val, err = scipy_integrate.quad(f, -30.0, 30.0, points=pts, limit=400,
                                        epsabs=0, epsrel=1e-12)
        ref = a / math.pi * val
        h, _ = oracle.voigt_H(a, u)
        assert abs(h - ref) <= 1e-5 * ref, (a, u, h, ref)
