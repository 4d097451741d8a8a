"""Seeded synthetic line lists and workload definitions.

These stand in for the HITRAN/HITEMP line lists the paper reads (Sec. 2.3,
Sec. 3), which are not available here.  This module only draws random
numbers and states workload parameters; it holds none of the method's
arithmetic, so the CUDA path and the CPU oracle can both consume it.

Workloads (all lines sorted by nu0; generator numpy default_rng(seed)):

  "small"     1e4 lines, nu0 ~ U(0, 3000) cm^-1, log10 S ~ U(-26, -19),
              gamma ~ U(0.02, 0.1) cm^-1/atm; T 1500 K, P 1 atm, 18 amu;
              grid 0..3000 at 0.01 (3e5 points); cutoff 25 cm^-1;
              10 k-bins, 20 Chebyshev coefficients.
  "medium"    1e5 lines over 0..30000 cm^-1, same distributions; grid
              3e6 points at 0.01; cutoff 100 cm^-1; 300 bins, 20 coeffs.
  "tp_grid"   1e6 lines, log10 S ~ N(-24, 3) redrawn into [-30, -18],
              E'' ~ U(0, 1e4) cm^-1; 8 T in linspace(500, 3000) x 8 P in
              logspace(-5, 2) bar (converted to atm); cutoff
              min(500 Gamma_L, 100 cm^-1); grid 3e6 points; 300 bins.
  "surrogate" 1e7 lines as tp_grid at 1500 K, 1 atm.
  "mixed"     4 species x 2.5e7 lines (masses 18, 16, 44, 17 amu), grid
              3e7 points at 0.001, 4 T x 4 P, 1000 bins.
"""
import numpy as np

SEED_BASE = 150303806
BAR_PER_ATM = 1.01325


def _rng(cfg, species=0):
    return np.random.default_rng(SEED_BASE + cfg + 1000 * species)


def draw_lines(n, nu_lo, nu_hi, rng, strengths="loguniform", with_elower=False):
    """Draw n lines; returns a dict of float64 arrays sorted by nu0."""
    nu0 = rng.uniform(nu_lo, nu_hi, size=n)
    if strengths == "loguniform":
        logS = rng.uniform(-26.0, -19.0, size=n)
    else:  # log-normal, sigma = 3 decades, redrawn into [-30, -18]
        logS = rng.normal(-24.0, 3.0, size=n)
        bad = (logS < -30.0) | (logS > -18.0)
        while bad.any():
            logS[bad] = rng.normal(-24.0, 3.0, size=int(bad.sum()))
            bad = (logS < -30.0) | (logS > -18.0)
    S0 = 10.0 ** logS
    gamma = rng.uniform(0.02, 0.1, size=n)
    out = {"nu0": nu0, "S0": S0, "gamma_air": gamma}
    if with_elower:
        out["E_lower"] = rng.uniform(0.0, 1.0e4, size=n)
    order = np.argsort(nu0, kind="stable")
    return {k: np.ascontiguousarray(v[order]) for k, v in out.items()}


# Workload table.  cut: ("abs", C) or ("lorentz", multiple, cap).
WORKLOADS = {
    "small": dict(cfg=1, nlines=10_000, nu_range=(0.0, 3000.0),
                  strengths="loguniform", elower=False, mass=18.0,
                  T=[1500.0], P_atm=[1.0], nu_min=0.0, dnu=0.01,
                  ngrid=300_000, cut=("abs", 25.0), nbins=10, ncheb=20),
    "medium": dict(cfg=2, nlines=100_000, nu_range=(0.0, 30000.0),
                   strengths="loguniform", elower=False, mass=18.0,
                   T=[1500.0], P_atm=[1.0], nu_min=0.0, dnu=0.01,
                   ngrid=3_000_000, cut=("abs", 100.0), nbins=300, ncheb=20),
    "tp_grid": dict(cfg=3, nlines=1_000_000, nu_range=(0.0, 30000.0),
                    strengths="lognormal", elower=True, mass=18.0,
                    T=list(np.linspace(500.0, 3000.0, 8)),
                    P_atm=list(np.logspace(-5.0, 2.0, 8) / BAR_PER_ATM),
                    nu_min=0.0, dnu=0.01, ngrid=3_000_000,
                    cut=("lorentz", 500.0, 100.0), nbins=300, ncheb=20),
    "surrogate": dict(cfg=4, nlines=10_000_000, nu_range=(0.0, 30000.0),
                      strengths="lognormal", elower=True, mass=18.0,
                      T=[1500.0], P_atm=[1.0], nu_min=0.0, dnu=0.01,
                      ngrid=3_000_000, cut=("lorentz", 500.0, 100.0),
                      nbins=300, ncheb=20),
    "mixed": dict(cfg=5, nlines=25_000_000, nu_range=(0.0, 30000.0),
                  strengths="lognormal", elower=True,
                  species_mass=[18.0, 16.0, 44.0, 17.0],
                  mixing=[0.25, 0.25, 0.25, 0.25],
                  T=list(np.linspace(500.0, 3000.0, 4)),
                  P_atm=list(np.logspace(-4.0, 2.0, 4) / BAR_PER_ATM),
                  nu_min=0.0, dnu=0.001, ngrid=30_000_000,
                  cut=("lorentz", 500.0, 100.0), nbins=1000, ncheb=20),
}


def workload_lines(name, nlines=None, species=0):
    """Line list of a named workload (optionally truncated to nlines draws)."""
    w = WORKLOADS[name]
    n = w["nlines"] if nlines is None else int(nlines)
    return draw_lines(n, w["nu_range"][0], w["nu_range"][1],
                      _rng(w["cfg"], species), w["strengths"], w["elower"])


def random_lines(n, seed, nu_lo=0.0, nu_hi=100.0, with_elower=False,
                 strengths="loguniform", extra_fields=False):
    """Small seeded line lists for tests.  extra_fields adds gamma_self,
    n_coll and delta drawn from plausible ranges."""
    rng = np.random.default_rng(seed)
    out = draw_lines(n, nu_lo, nu_hi, rng, strengths, with_elower)
    if extra_fields:
        out["gamma_self"] = rng.uniform(0.05, 0.5, size=n)
        out["n_coll"] = rng.uniform(0.3, 0.9, size=n)
        out["delta"] = rng.uniform(-0.02, 0.02, size=n)
    return out


def uniform_kappa(n, seed, decades=12):
    """Positive, log-uniform opacity-like values for k-distribution tests."""
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.uniform(-20.0 - decades, -20.0, size=n)
