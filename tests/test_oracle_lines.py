"""Pins of the oracle's line preparation and opacity accumulation
(Sec. 2.3-2.4): hand values, brute-force windows and counts, profile
normalisation, linearity, thread independence."""
import math

import numpy as np
import pytest

import oracle
from paper_1503_03806_gb300 import synth

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(f"{GOLDEN}/{name}") as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def test_doppler_width_hand_value():
    g = _golden("lineprep_hand_values.txt")
    lines = {"nu0": np.array([1000.0, 20000.0]), "S0": np.array([1e-20, 1e-20]),
             "gamma_air": np.array([0.05, 0.05])}
    cond = oracle.Condition(1500.0, 1.0, 18.0, 0.0, 0.01, 10, oracle.CUT_ABS, 1.0)
    r = oracle.lineprep(lines, cond)
    np.testing.assert_allclose(r["gD"] / lines["nu0"], g["gammaD_over_nu0_1500K_18amu"],
                               rtol=2e-6)
    # Gamma_L = gamma P (T0/T)^0.5 with gamma_self = gamma_air (Sec. 2.3)
    np.testing.assert_allclose(r["gL"], 0.05 * math.sqrt(296.0 / 1500.0), rtol=1e-15)
    # damping and scale parameters (Sec. 2.3)
    np.testing.assert_allclose(r["a"], math.sqrt(math.log(2)) * r["gL"] / r["gD"], rtol=1e-15)
    np.testing.assert_allclose(r["Sp"], 1e-20 * math.sqrt(math.log(2) / math.pi) / r["gD"],
                               rtol=1e-15)


def test_strength_scaling_invariants():
    # S/S0 = (Q0/Q) exp(-c2E''(1/T-1/T0)) (1-e^{-c2 nu/T})/(1-e^{-c2 nu/T0})
    n = 50
    rng = np.random.default_rng(5)
    lines = {"nu0": np.sort(rng.uniform(10, 20000, n)), "S0": 10 ** rng.uniform(-26, -19, n),
             "gamma_air": np.full(n, 0.05), "E_lower": rng.uniform(0, 1e4, n)}
    # at T = T0 and Q ratio 1, nothing changes
    r0 = oracle.lineprep(lines, oracle.Condition(296.0, 1.0, 18.0, 0.0, 0.01, 10, q_ratio=1.0))
    np.testing.assert_allclose(r0["S"], lines["S0"], rtol=1e-14)
    # the Q ratio enters linearly
    r1 = oracle.lineprep(lines, oracle.Condition(900.0, 1.0, 18.0, 0.0, 0.01, 10, q_ratio=1.0))
    r2 = oracle.lineprep(lines, oracle.Condition(900.0, 1.0, 18.0, 0.0, 0.01, 10, q_ratio=0.37))
    np.testing.assert_allclose(r2["S"], 0.37 * r1["S"], rtol=1e-14)
    # Boltzmann factor: with E'' shifted by dE the ratio is exp(-c2 dE (1/T - 1/T0)),
    # c2 = h c / k_B = 1.4387768775 cm K (CODATA 2018 exact)
    g = _golden("lineprep_hand_values.txt")
    lines2 = dict(lines)
    lines2["E_lower"] = lines["E_lower"] + 1000.0
    r3 = oracle.lineprep(lines2, oracle.Condition(900.0, 1.0, 18.0, 0.0, 0.01, 10, q_ratio=1.0))
    np.testing.assert_allclose(r3["S"] / r1["S"], g["boltzmann_ratio_dE1000_900K"], rtol=1e-12)


def test_pressure_shift_and_general_broadening():
    lines = synth.random_lines(40, 9, 100.0, 200.0, extra_fields=True)
    cond = oracle.Condition(800.0, 2.5, 18.0, 0.0, 0.01, 100, oracle.CUT_ABS, 1.0)
    r = oracle.lineprep(lines, cond)
    np.testing.assert_allclose(r["nu0p"], lines["nu0"] + lines["delta"] * 2.5, rtol=1e-15)
    ref = (296.0 / 800.0) ** lines["n_coll"] * (lines["gamma_air"] * 1.25 + lines["gamma_self"] * 1.25)
    np.testing.assert_allclose(r["gL"], ref, rtol=1e-14)


def _bruteforce_window(nu0p, cut, nu_min, dnu, ngrid):
    i = np.arange(ngrid)
    nu = nu_min + i * dnu
    d = np.abs(nu - nu0p)
    inside = d <= cut * (1 - 1e-12)
    outside = d > cut * (1 + 1e-12)
    return i[inside], i[outside]


@pytest.mark.parametrize("kind", [oracle.CUT_ABS, oracle.CUT_LORENTZ, oracle.CUT_NONE])
def test_window_bounds_bruteforce(kind):
    lines = synth.random_lines(60, 11, -3.0, 103.0)
    cond = oracle.Condition(1500.0, 1.0, 18.0, 0.0, 0.01, 10000, kind,
                            {0: 2.5, 1: 40.0, 2: 0.0}[kind], 1.5)
    r = oracle.lineprep(lines, cond)
    for l in range(60):
        lo, hi = r["ilo"][l], r["ihi"][l]
        if kind == oracle.CUT_NONE:
            assert lo == 0 and hi == 9999
            continue
        ins, outs = _bruteforce_window(r["nu0p"][l], r["gL"][l] * 40.0 if kind == 1 else 2.5,
                                       0.0, 0.01, 10000)
        if kind == oracle.CUT_LORENTZ:
            cut = min(40.0 * r["gL"][l], 1.5)
            ins, outs = _bruteforce_window(r["nu0p"][l], cut, 0.0, 0.01, 10000)
        if ins.size:
            assert lo <= ins.min() and hi >= ins.max()
        assert not np.any((outs >= lo) & (outs <= hi))


def _small_cond(kind=oracle.CUT_ABS, cut=2.0, ngrid=20000, T=1500.0, P=1.0):
    return oracle.Condition(T, P, 18.0, 0.0, 0.01, ngrid, kind, cut, 1.0)


def test_single_line_equals_Sp_times_H():
    lines = {"nu0": np.array([50.003]), "S0": np.array([3e-21]), "gamma_air": np.array([0.07])}
    cond = _small_cond(cut=3.0, ngrid=10000)
    kap, ev, reg = oracle.opacity(lines, cond)
    r = oracle.lineprep(lines, cond)
    assert ev == r["ihi"][0] - r["ilo"][0] + 1
    for i in range(int(r["ilo"][0]), int(r["ihi"][0]) + 1, 37):
        nu_i = 0.0 + i * 0.01
        u = (nu_i - r["nu0p"][0]) * r["ku"][0]
        assert kap[i] == r["Sp"][0] * oracle.voigt_H(r["a"][0], u)[0]
    assert kap[: r["ilo"][0]].sum() == 0 and kap[r["ihi"][0] + 1:].sum() == 0


def test_profile_is_normalised():
    # sum_i Phi(nu_i) dnu = 1 (Sec. 2.3) on a fine grid without cutoff, with the
    # Lorentzian tails beyond the grid added analytically.
    S = 1.0
    lines = {"nu0": np.array([1000.0]), "S0": np.array([S]), "gamma_air": np.array([0.02])}
    dnu = 0.0001
    half = 30.0
    ngrid = int(2 * half / dnu) + 1
    cond = oracle.Condition(1500.0, 1.0, 18.0, 1000.0 - half, dnu, ngrid, oracle.CUT_NONE, 0.0)
    kap, ev, reg = oracle.opacity(lines, cond, nthreads=4)
    gL = oracle.lineprep(lines, cond)["gL"][0]
    tails = 2.0 * (0.5 - math.atan(half / gL) / math.pi)
    total = kap.sum() * dnu + tails
    assert abs(total - 1.0) < 2e-5, total
    assert reg[0] > 0 and reg[1] > 0 and reg[2] > 0


def test_linearity_and_thread_independence():
    lines = synth.random_lines(300, 21, 0.0, 200.0)
    cond = _small_cond(cut=5.0, ngrid=20000)
    k_all, ev_all, _ = oracle.opacity(lines, cond, nthreads=1)
    k_mt, ev_mt, _ = oracle.opacity(lines, cond, nthreads=5)
    assert np.array_equal(k_all, k_mt) and ev_all == ev_mt
    A = {k: v[::2] for k, v in lines.items()}
    B = {k: v[1::2] for k, v in lines.items()}
    kA, evA, _ = oracle.opacity(A, cond)
    kB, evB, _ = oracle.opacity(B, cond)
    assert evA + evB == ev_all
    np.testing.assert_allclose(kA + kB, k_all, rtol=1e-13, atol=0)
    # weight and accumulate
    k2, _, _ = oracle.opacity(B, cond, weight=0.25, kappa=kA)
    np.testing.assert_allclose(k2, kA + 0.25 * kB, rtol=1e-15)


def test_eval_count_bruteforce():
    lines = synth.random_lines(100, 31, 0.0, 100.0)
    cond = _small_cond(cut=1.7, ngrid=10000)
    _, ev, _ = oracle.opacity(lines, cond)
    r = oracle.lineprep(lines, cond)
    assert ev == int(np.maximum(r["ihi"] - r["ilo"] + 1, 0).sum())
    nu = np.arange(10000) * 0.01
    brute = sum(int(np.sum(np.abs(nu - c) <= 1.7 * (1 - 1e-12))) for c in r["nu0p"])
    brute_hi = sum(int(np.sum(np.abs(nu - c) <= 1.7 * (1 + 1e-12))) for c in r["nu0p"])
    assert brute <= ev <= brute_hi


def test_points_equal_full_grid():
    lines = synth.random_lines(200, 41, 0.0, 100.0, with_elower=True)
    cond = oracle.Condition(2000.0, 0.3, 18.0, 0.0, 0.01, 10000, oracle.CUT_LORENTZ, 500.0, 3.0,
                            q_ratio=0.5)
    k, ev, _ = oracle.opacity(lines, cond)
    idx = np.array([0, 17, 555, 4321, 9999, 5000])
    kp, _ = oracle.opacity_points(lines, cond, idx)
    assert np.array_equal(kp, k[idx])


def test_per_line_mass_and_weight():
    # one list holding two species (Sec. 2.1: abundance-weighted opacities are
    # added before the k-distribution)
    A = synth.random_lines(150, 51, 0.0, 100.0)
    B = synth.random_lines(120, 52, 0.0, 100.0)
    cond = _small_cond(cut=4.0, ngrid=10000)
    kA, _, _ = oracle.opacity(A, oracle.Condition(1500.0, 1.0, 18.0, 0.0, 0.01, 10000,
                                                  oracle.CUT_ABS, 4.0))
    kB, _, _ = oracle.opacity(B, oracle.Condition(1500.0, 1.0, 44.0, 0.0, 0.01, 10000,
                                                  oracle.CUT_ABS, 4.0))
    mix = {k: np.concatenate([A[k], B[k]]) for k in A}
    mix["mass"] = np.concatenate([np.full(150, 18.0), np.full(120, 44.0)])
    mix["weight"] = np.concatenate([np.full(150, 0.7), np.full(120, 0.3)])
    kM, _, _ = oracle.opacity(mix, cond)
    np.testing.assert_allclose(kM, 0.7 * kA + 0.3 * kB, rtol=1e-13, atol=0)
    # Doppler width scales as m^-1/2
    r = oracle.lineprep(mix, cond)
    one = {k: v[:1] for k, v in A.items()}
    one4 = dict(one, mass=np.array([72.0]))
    g18 = oracle.lineprep(one, oracle.Condition(1500.0, 1.0, 18.0, 0.0, 0.01, 10))["gD"][0]
    g72 = oracle.lineprep(one4, oracle.Condition(1500.0, 1.0, 18.0, 0.0, 0.01, 10))["gD"][0]
    assert abs(g18 / g72 - 2.0) < 1e-15
    assert np.all(r["gD"][:150] > 0)
