"""Pins of the oracle's k-distribution stage (Sec. 2.1-2.2, 2.6): sort by a
library sort, Chebyshev fit by exact recovery and numpy's chebfit, the
Lebesgue/Riemann invariants of Sec. 2.1."""
import numpy as np

import oracle
from paper_1503_03806_gb300 import synth


def test_sort_bins_matches_numpy():
    k = synth.uniform_kappa(12 * 997, 1)
    k[5] = k[6] = k[100]  # ties
    s = oracle.sort_bins(k, 12)
    ref = np.sort(k.reshape(12, -1), axis=1).ravel()
    assert np.array_equal(s, ref)


def _cheb_design(nb, ncheb):
    g = (np.arange(nb) + 0.5) / nb
    return np.polynomial.chebyshev.chebvander(2 * g - 1, ncheb - 1)


def test_chebfit_recovers_low_degree_series():
    # ln k(g) = sum_k c_k T_k(2g-1) exactly -> LS fit returns c (Sec. 2.6)
    rng = np.random.default_rng(2)
    nb, ncheb, nbins = 3000, 20, 4
    c_true = rng.normal(0, 1, (nbins, ncheb)) / (1 + np.arange(ncheb)) ** 2
    c_true[:, 0] -= 45.0
    A = _cheb_design(nb, ncheb)
    L = (A @ c_true.T).T
    k = np.exp(L).ravel()
    coef, mean = oracle.chebfit(k, nbins, ncheb)
    assert np.max(np.abs(coef - c_true)) < 1e-10 * np.max(np.abs(c_true))
    np.testing.assert_allclose(mean, k.reshape(nbins, nb).mean(axis=1), rtol=1e-13)


def test_chebfit_matches_numpy_chebfit():
    nbins, nb, ncheb = 5, 2000, 20
    k = np.sort(synth.uniform_kappa(nbins * nb, 7).reshape(nbins, nb), axis=1)
    coef, _ = oracle.chebfit(k.ravel(), nbins, ncheb)
    g = (np.arange(nb) + 0.5) / nb
    for b in range(nbins):
        ref = np.polynomial.chebyshev.chebfit(2 * g - 1, np.log(k[b]), ncheb - 1)
        assert np.max(np.abs(coef[b] - ref)) < 1e-10 * np.max(np.abs(ref))


def test_kappa_floor():
    nb = 100
    k = np.zeros(nb)
    k[50:] = 1e-10
    coef, _ = oracle.chebfit(k, 1, 4, kappa_floor=1e-30)
    g = (np.arange(nb) + 0.5) / nb
    ref = np.polynomial.chebyshev.chebfit(2 * g - 1, np.log(np.maximum(k, 1e-30)), 3)
    np.testing.assert_allclose(coef[0], ref, rtol=1e-9, atol=1e-9)


def test_chebeval_inverts_fit():
    c = np.array([-40.0, 2.0, -0.3, 0.05])
    g = np.linspace(0.01, 0.99, 7)
    ref = np.exp(np.polynomial.chebyshev.chebval(2 * g - 1, c))
    np.testing.assert_allclose(oracle.chebeval(c, g), ref, rtol=1e-14)


def _opacity_kappa(nbins, seed=3):
    lines = synth.random_lines(400, seed, 0.0, 100.0)
    cond = oracle.Condition(1500.0, 1.0, 18.0, 0.0, 0.01, 10000, oracle.CUT_ABS, 10.0)
    k, _, _ = oracle.opacity(lines, cond, nthreads=4)
    return k


def test_transmission_lebesgue_equals_riemann():
    # Sec. 2.1: int F dx = int F dy with F = exp(-kappa m): the band-mean
    # transmission of the unsorted bin equals the integral over g of the
    # sorted k(g) (midpoint rule), up to summation order.
    nbins = 10
    k = _opacity_kappa(nbins)
    s = oracle.sort_bins(k, nbins)
    m = np.logspace(14, 24, 11)
    direct, _ = oracle.transmission(s, nbins, m)
    riemann = np.exp(-np.outer(k, m)).reshape(nbins, -1, m.size).mean(axis=1)
    np.testing.assert_allclose(direct, riemann, rtol=1e-12, atol=1e-300)
    # int kappa dx = int kappa dy (the bin mean)
    _, coef_mean = oracle.chebfit(s, nbins, 20)
    np.testing.assert_allclose(coef_mean, k.reshape(nbins, -1).mean(axis=1), rtol=1e-13)


def test_fit_transmission_close_to_direct():
    # Sec. 3.2: with N_nu >= 1e3 per bin, the 20-coefficient fit changes the
    # transmission by << 1 % at every column mass.
    nbins = 10
    k = _opacity_kappa(nbins, seed=8)
    s, coef, _ = oracle.kdist(k, nbins, 20, kappa_floor=1e-250)
    m = np.logspace(12, 26, 29)
    direct, fit = oracle.transmission(s, nbins, m, coeffs=coef)
    assert np.max(np.abs(fit - direct)) < 1e-2
