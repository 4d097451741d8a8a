"""The FP32 form's Algorithm 916 series (Sec. 2.4 core region), as the core
kernel sums it: with h = 1/2 and d the offset of a window's first node from
x, each term's Gaussian factor splits as

    e^{-(d + t h)^2} = e^{-d^2} rho^t e^{-t^2/4},   rho = e^{-d},

so a window of weights w_t sums as e^{-d^2} times the polynomial
sum_t (e^{-t^2/4} w_t) rho^t, taken by Horner's rule from the last term.
The S2 series (nodes at nh + x) has offset d + 2x, so for a window starting
at n0 = 1 its ratio is rho e^{-2x} and its first factor e^{-d^2} e^{-2x}.

Checked here in FP64 against the terms summed one by one, over the points
where the kernel takes each path, and the kernel's table of e^{-t^2/4}
(read from the header) against the exponential rounded to FP32: a wrong
entry, a wrong sign of the offset or a wrong S2 ratio fails.
"""
import math
import os
import re

import numpy as np

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_1503_03806_gb300", "csrc", "voigt_core.cuh")
TERMS, S2_TERMS, TAIL = 18, 8, 4.3


def _window_start(x):
    return max(1, math.ceil((x - TAIL) * 2.0))


def _weights(y):
    return np.array([1.0 / ((0.5 * n) ** 2 + y * y) for n in range(1, 30)])


def _direct(x, y):
    # S3 and S2 term by term over the kernel's 18 (S3) and 8 (S2) nodes
    n0 = _window_start(x)
    w = _weights(y)
    s3 = sum(math.exp(-((n0 + t) * 0.5 - x) ** 2) * w[n0 - 1 + t] for t in range(TERMS))
    s2 = sum(math.exp(-((n0 + t) * 0.5 + x) ** 2) * w[n0 - 1 + t] for t in range(S2_TERMS))
    return s3, s2


def _horner(x, y, A):
    n0 = _window_start(x)
    w = _weights(y)[n0 - 1:]
    d = n0 * 0.5 - x
    rho3 = math.exp(-d)
    acc3 = 0.0
    for t in range(TERMS - 1, -1, -1):
        acc3 = rho3 * acc3 + A[t] * w[t]
    g = math.exp(-2.0 * x)
    rho2 = rho3 * g
    acc2 = 0.0
    for t in range(S2_TERMS - 1, -1, -1):
        acc2 = rho2 * acc2 + A[t] * w[t]
    E3 = math.exp(-d * d)
    return E3 * acc3, (E3 * g * acc2 if n0 == 1 else 0.0)


def _table():
    src = open(HEADER).read()
    m = re.search(r"A916_GAUSS_F32\[A916_TERMS_F32\]\s*=\s*\{([^}]*)\}", src)
    assert m, "table of e^{-t^2/4} not found"
    return [float.fromhex(v.strip().rstrip("f")) for v in m.group(1).split(",") if v.strip()]


def test_gaussian_factor_table():
    A = _table()
    assert len(A) == TERMS
    for t, v in enumerate(A):
        assert v == float(np.float32(math.exp(-t * t / 4.0))), t


def test_horner_form_equals_the_terms():
    A = [math.exp(-t * t / 4.0) for t in range(TERMS)]
    rng = np.random.default_rng(916)
    for _ in range(3000):
        while True:
            x, y = rng.uniform(0.0, 10.0), 10.0 ** rng.uniform(-6.0, 1.0)
            if x * x + y * y < 100.0:
                break
        s3, s2 = _direct(x, y)
        h3, h2 = _horner(x, y, A)
        assert abs(h3 - s3) <= 1e-13 * s3, (x, y)
        if _window_start(x) == 1:
            assert abs(h2 - s2) <= 1e-13 * s2 + 1e-300, (x, y)
        else:
            # the kernel leaves S2 out where the window starts past n = 1:
            # every S2 term there is below e^{-(1 + 4.8)^2} of its weight
            assert s2 <= math.exp(-33.0) * max(_weights(y)), (x, y)


def test_a_wrong_offset_sign_or_ratio_fails():
    A = [math.exp(-t * t / 4.0) for t in range(TERMS)]
    x, y = 2.7, 0.3
    s3, s2 = _direct(x, y)
    h3, h2 = _horner(x, y, A)
    assert abs(h3 - s3) <= 1e-13 * s3 and abs(h2 - s2) <= 1e-13 * s2
    # the same sums with rho = e^{+d}, or with S2's ratio taken as S3's
    n0 = _window_start(x)
    w = _weights(y)[n0 - 1:]
    d = n0 * 0.5 - x
    acc = 0.0
    for t in range(TERMS - 1, -1, -1):
        acc = math.exp(d) * acc + A[t] * w[t]
    assert abs(math.exp(-d * d) * acc - s3) > 1e-3 * s3
    acc = 0.0
    for t in range(S2_TERMS - 1, -1, -1):
        acc = math.exp(-d) * acc + A[t] * w[t]
    assert abs(math.exp(-d * d) * math.exp(-2.0 * x) * acc - s2) > 1e-3 * s2
