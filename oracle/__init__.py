"""FP64 CPU oracle for the HELIOS-K hot path (arXiv:1503.03806).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_1503_03806_gb300``), and neither imports
the other; both read the same seeded inputs from
``paper_1503_03806_gb300.synth``.

The arithmetic lives in ``helk_oracle.c`` (plain C, ``-ffp-contract=off``).
This module is argument marshalling with ctypes plus a numpy FP64 reference
of the Voigt-surrogate MLP (``mlp_*``).

Pins (tests/test_oracle_*.py), each independent of the formula it checks:
  or_K916      mpmath w(z) to <= 1e-13 rel over the core region; erfcx(y) at
               x = 0 (scipy); exp(-x^2) at y = 0; evenness in x.
  or_gh3/gh1   the same sums in mpmath at 50 digits; error vs exact w(z)
               within the method's bound (<= 6e-6 / 2e-6); GH1 = Lorentz wing.
  voigt_H      profile normalisation sum Phi dnu = 1; Gaussian (x) Lorentzian
               convolution by scipy quad; region boundaries.
  lineprep     hand values (Gamma_D/nu0 = 3.26914e-6 at 1500 K, 18 amu),
               T = T0 leaves S unchanged, window bounds by brute force.
  opacity      single line = S' H, linearity in the line list, eval counts by
               brute force, thread-count independence.
  sort         numpy.sort per bin (permutation + monotone).
  chebfit      exact recovery of degree < n Chebyshev series; agreement with
               numpy.polynomial.chebyshev.chebfit.
  transmission band-mean transmission = integral over g (Sec. 2.1, Eq. for T).
  mlp          finite differences of the loss.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

CUT_ABS, CUT_LORENTZ, CUT_NONE = 0, 1, 2

_d = ctypes.c_double
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_p = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        # HELK_ORACLE_LIB: a deliberately broken build of the oracle, used by
        # tests/test_oracle_mutations.py to show that the pins catch mistakes
        path = os.environ.get("HELK_ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        L.or_K916.restype = _d
        L.or_K916.argtypes = [_d, _d]
        L.or_gh3.restype = _d
        L.or_gh3.argtypes = [_d, _d]
        L.or_gh1.restype = _d
        L.or_gh1.argtypes = [_d, _d]
        L.or_voigt_H.restype = _d
        L.or_voigt_H.argtypes = [_d, _d, _p]
        line_args = [_i64] + [_p] * 9 + [_d, _d, _d, _d, ctypes.c_int, _d, _d,
                                         _d, _d, _i64]
        L.or_lineprep.restype = ctypes.c_int
        L.or_lineprep.argtypes = line_args + [_p] * 9
        L.or_opacity.restype = ctypes.c_int
        L.or_opacity.argtypes = line_args + [_d, ctypes.c_int, _p,
                                             ctypes.c_int, _p, _p]
        L.or_opacity_points.restype = ctypes.c_int
        L.or_opacity_points.argtypes = line_args + [_i64, _p, _p, _p]
        L.or_sort_bins.restype = ctypes.c_int
        L.or_sort_bins.argtypes = [_p, _i64, _i32, _p]
        L.or_chebfit.restype = ctypes.c_int
        L.or_chebfit.argtypes = [_p, _i64, _i32, _i32, _d, _p, _p]
        L.or_chebeval.restype = ctypes.c_int
        L.or_chebeval.argtypes = [_p, _i32, _i64, _p, _p]
        L.or_transmission.restype = ctypes.c_int
        L.or_transmission.argtypes = [_p, _i64, _i32, _p, _i32, _i64, _i32,
                                      _p, _p, _p]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- Voigt ----
def K916(x, y):
    """Algorithm 916 core, Re w(x+iy) (Sec. 2.4)."""
    return lib().or_K916(float(x), float(y))


def gh3(x, y):
    """3-node Gauss-Hermite Voigt (Sec. 2.4)."""
    return lib().or_gh3(float(x), float(y))


def gh1(x, y):
    """1-node Gauss-Hermite Voigt = Lorentz far wing (Sec. 2.4)."""
    return lib().or_gh1(float(x), float(y))


def voigt_H(a, u):
    """Region-dispatched H_V(a, u); returns (H, region) with region 0 = 916,
    1 = GH3, 2 = GH1 (Sec. 2.4)."""
    reg = ctypes.c_int(0)
    h = lib().or_voigt_H(float(a), float(u), ctypes.byref(reg))
    return h, reg.value


# ------------------------------------------------------------ line list ----
class Condition:
    """One (T, P) condition with its grid and cutoff.

    T [K], P [atm], mass [amu], q_ratio = Q(T0)/Q(T) (used only when the line
    list has lower-state energies), cutoff kind/value/cap as in Sec. 2.4,
    grid nu_i = nu_min + i*dnu for i < ngrid.
    """

    def __init__(self, T, P, mass, nu_min, dnu, ngrid, cut_kind=CUT_ABS,
                 cut_value=25.0, cut_cap=0.0, q_ratio=1.0):
        self.T, self.P, self.mass, self.q_ratio = float(T), float(P), float(mass), float(q_ratio)
        self.nu_min, self.dnu, self.ngrid = float(nu_min), float(dnu), int(ngrid)
        self.cut_kind, self.cut_value, self.cut_cap = int(cut_kind), float(cut_value), float(cut_cap)

    def args(self):
        return [self.T, self.P, self.mass, self.q_ratio, self.cut_kind,
                self.cut_value, self.cut_cap, self.nu_min, self.dnu, self.ngrid]


LINE_FIELDS = ("nu0", "S0", "E_lower", "gamma_air", "gamma_self", "n_coll", "delta", "mass",
               "weight")


def _line_ptrs(lines):
    keep = {k: _f64(lines.get(k)) for k in LINE_FIELDS}
    n = int(keep["nu0"].shape[0])
    ptrs = [_ptr(keep[k]) for k in LINE_FIELDS]
    return n, ptrs, keep


def lineprep(lines, cond):
    """Per-line records at one condition (Sec. 2.3-2.4)."""
    n, ptrs, keep = _line_ptrs(lines)
    out = {k: np.empty(n) for k in ("nu0p", "S", "Sp", "ku", "a", "gD", "gL")}
    out["ilo"] = np.empty(n, dtype=np.int64)
    out["ihi"] = np.empty(n, dtype=np.int64)
    rc = lib().or_lineprep(n, *ptrs, *cond.args(),
                           *[_ptr(out[k]) for k in ("nu0p", "S", "Sp", "ku", "a",
                                                    "gD", "gL", "ilo", "ihi")])
    assert rc == 0
    return out


def opacity(lines, cond, weight=1.0, kappa=None, nthreads=1):
    """kappa on the full grid; returns (kappa, evals, region_counts)."""
    n, ptrs, keep = _line_ptrs(lines)
    acc = kappa is not None
    if kappa is None:
        kappa = np.zeros(cond.ngrid)
    else:
        kappa = np.ascontiguousarray(kappa, dtype=np.float64).copy()
    ev = np.zeros(1, dtype=np.int64)
    reg = np.zeros(3, dtype=np.int64)
    rc = lib().or_opacity(n, *ptrs, *cond.args(), float(weight), int(acc),
                          _ptr(kappa), int(nthreads), _ptr(ev), _ptr(reg))
    assert rc == 0
    return kappa, int(ev[0]), reg


def opacity_points(lines, cond, idx):
    """kappa at the grid indices idx only; returns (kappa_pts, evals)."""
    n, ptrs, keep = _line_ptrs(lines)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(idx.shape[0])
    ev = np.zeros(1, dtype=np.int64)
    rc = lib().or_opacity_points(n, *ptrs, *cond.args(), idx.shape[0],
                                 _ptr(idx), _ptr(out), _ptr(ev))
    assert rc == 0
    return out, int(ev[0])


# --------------------------------------------------------- k-distribution --
def sort_bins(kappa, nbins):
    kappa = _f64(kappa)
    out = np.empty_like(kappa)
    assert lib().or_sort_bins(_ptr(kappa), kappa.shape[0], int(nbins), _ptr(out)) == 0
    return out


def chebfit(sorted_kappa, nbins, ncheb, kappa_floor=1e-250):
    """Per-bin Chebyshev coefficients (nbins, ncheb) and bin means."""
    s = _f64(sorted_kappa)
    coef = np.empty((nbins, ncheb))
    mean = np.empty(nbins)
    rc = lib().or_chebfit(_ptr(s), s.shape[0], int(nbins), int(ncheb),
                          float(kappa_floor), _ptr(coef), _ptr(mean))
    assert rc == 0, rc
    return coef, mean


def chebeval(coef, g):
    coef = _f64(coef)
    g = _f64(g)
    out = np.empty_like(g)
    lib().or_chebeval(_ptr(coef), coef.shape[0], g.shape[0], _ptr(g), _ptr(out))
    return out


def kdist(kappa, nbins, ncheb, kappa_floor=1e-250):
    """Sort + fit; returns (sorted, coeffs, mean)."""
    s = sort_bins(kappa, nbins)
    c, m = chebfit(s, nbins, ncheb, kappa_floor)
    return s, c, m


def transmission(sorted_kappa, nbins, m, coeffs=None, ng=None):
    """Per-bin transmission T_b(m) from the samples and (optionally) the fit."""
    s = _f64(sorted_kappa)
    m = _f64(np.atleast_1d(m))
    nm = m.shape[0]
    direct = np.empty((nbins, nm))
    fit = np.empty((nbins, nm)) if coeffs is not None else None
    ncheb = 0 if coeffs is None else int(np.asarray(coeffs).shape[1])
    cf = None if coeffs is None else _f64(coeffs)
    if ng is None:
        ng = s.shape[0] // nbins
    rc = lib().or_transmission(_ptr(s), s.shape[0], int(nbins), _ptr(cf), ncheb,
                               int(ng), nm, _ptr(m), _ptr(direct), _ptr(fit))
    assert rc == 0
    return direct, fit
