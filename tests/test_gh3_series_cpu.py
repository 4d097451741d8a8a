"""The FP32 form's expansion of the 3-node Gauss-Hermite term in t = 1/r^2
(Sec. 2.4 method regions; used on whole warp spans far from the line
centre): on the region where the kernels take it (r^2 >= R_s, R_s >= 1000,
R_s^3 >= 1.25^3 5e7 (7.875 + 15 a^2)), the series truncated after its third
coefficient stays within 1.1e-8 of the exact quadrature term for every a.

The exact term is the 3-node rule itself -- weights 4 w1 at u and w1 at
u -+ t0 (t0^2 = 3/2) of the Lorentzian a / (pi ((u - x)^2 + a^2)) -- and the
series coefficients are the kernel's g0 = 3 P, g1 = 4.5 P,
g2 = (11.25 - 6 a^2) P with P the line's factor, so a wrong coefficient, a
wrong sign or a threshold set too low fails here.
"""
import numpy as np


def _exact_over_P(u2, a2):
    # three Lorentzian nodes, normalised so that the series' P factor is 1:
    # (4 / r2 + 1 / ((u - t0)^2 + a^2) + 1 / ((u + t0)^2 + a^2)) / 2,
    # which is the kernel's n / (r2 p) for P3h = 1
    u = np.sqrt(u2)
    t0 = np.sqrt(1.5)
    r2 = u2 + a2
    return (4.0 / r2 + 1.0 / ((u - t0) ** 2 + a2) + 1.0 / ((u + t0) ** 2 + a2)) / 2.0


def _series_over_P(r2, a2):
    t = 1.0 / r2
    return t * (3.0 + t * (4.5 + t * (11.25 - 6.0 * a2)))


def _holds(r2, a2):
    return (r2 >= 1000.0) & (r2 ** 3 >= 9.765625e7 * (15.0 * a2 + 7.875))


def test_leading_terms_match_the_quadrature():
    # far from the centre the term tends to 3 P / r2 (all nodes at weight sum 6 w1)
    for a2 in (0.0, 1.0, 50.0):
        r2 = np.array([1e8, 1e10])
        ex = _exact_over_P(r2 - a2, a2)
        assert np.allclose(ex * r2, 3.0, rtol=1e-6)


def test_series_within_bound_where_taken():
    worst = 0.0
    for a2 in np.concatenate([[0.0, 1e-8, 1e-4, 0.01, 0.1], np.logspace(-1, 5.99, 300)]):
        r2 = np.logspace(np.log10(max(100.0, a2)), 6.0, 1500)
        r2 = r2[_holds(r2, a2) & (r2 > a2)]
        if r2.size == 0:
            continue
        ex = _exact_over_P(r2 - a2, a2)
        err = np.max(np.abs(_series_over_P(r2, a2) / ex - 1.0))
        worst = max(worst, err)
    assert worst < 1.1e-8, worst


def test_threshold_is_needed():
    # just below the threshold at large a the truncation is visible: the
    # condition is not slack enough to be dropped
    a2 = 1.0e4
    r2 = np.logspace(np.log10(a2 * 1.01), 6.0, 4000)
    below = r2[~_holds(r2, a2)]
    ex = _exact_over_P(below - a2, a2)
    assert np.max(np.abs(_series_over_P(below, a2) / ex - 1.0)) > 1.1e-8
