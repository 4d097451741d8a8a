"""Shared helpers for the parity tests: one description of a condition that
both the oracle and the CUDA binding accept."""
import os

import numpy as np

import oracle

CUT_KIND = {"abs": oracle.CUT_ABS, "lorentz": oracle.CUT_LORENTZ, "none": oracle.CUT_NONE}
NTHREADS = max(1, min(32, os.cpu_count() or 1))


class Case:
    def __init__(self, T, P, mass, grid, cut, q_ratio=1.0):
        self.T, self.P, self.mass, self.grid, self.cut, self.q_ratio = T, P, mass, grid, cut, q_ratio

    def oracle_cond(self):
        kind = CUT_KIND[self.cut[0]]
        value = self.cut[1] if len(self.cut) > 1 else 0.0
        cap = self.cut[2] if len(self.cut) > 2 else 0.0
        return oracle.Condition(self.T, self.P, self.mass, self.grid[0], self.grid[1], self.grid[2],
                                kind, value, cap, q_ratio=self.q_ratio)

    def gpu(self, ctx, **kw):
        return ctx.opacity(self.T, self.P, self.mass, self.cut, self.grid, q_ratio=self.q_ratio, **kw)


def workload_case(w, T=None, P=None, mass=None):
    return Case(w["T"][0] if T is None else T, w["P_atm"][0] if P is None else P,
                w.get("mass", 18.0) if mass is None else mass,
                (w["nu_min"], w["dnu"], w["ngrid"]), w["cut"])


def assert_rel(got, ref, rtol, what=""):
    """Element-wise |got - ref| <= rtol |ref|; exact zeros must match."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape
    zero = ref == 0
    assert np.all(got[zero] == 0), "%s: nonzero where the oracle is 0" % what
    nz = ~zero
    if nz.any():
        rel = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
        worst = float(rel.max())
        assert worst <= rtol, "%s: max rel err %.3e > %.1e at %d" % (
            what, worst, rtol, int(np.flatnonzero(nz)[rel.argmax()]))
        return worst
    return 0.0


def near_lines(lines, nu_lo, nu_hi, reach):
    """The lines whose centre lies in [nu_lo - reach, nu_hi + reach] (a list
    sorted by nu0): with reach at least the largest window half-width, no
    other line reaches a grid point in [nu_lo, nu_hi]."""
    a, b = np.searchsorted(lines["nu0"], [nu_lo - reach, nu_hi + reach])
    return {k: np.ascontiguousarray(v[a:b]) for k, v in lines.items()}


def check_sampled_f32(k_row, nbins, idx, oracle_at, rtol=1e-5, floor=1e-8, what=""):
    """FP32 parity of one condition's device result k_row (numpy, the whole
    grid) on sampled grid indices idx, with every threshold taken from the
    oracle, never from the device result.

    For each k-bin the sample touches, the device's largest value in the bin
    is checked too, so a device value inflated anywhere in a touched bin
    fails (it becomes the bin's argmax).  The bin's floor is `floor` times the
    largest oracle value among its checked points (the samples and the device
    argmax; when the device is right, the argmax is the bin's largest
    point).  Points above the floor must agree to rtol relative; points below
    it to rtol times the floor, absolutely.  oracle_at(indices) returns the
    oracle's values at sorted unique grid indices.  Returns the worst
    relative error above the floor."""
    n = k_row.shape[0]
    nb = n // nbins
    bins = np.unique(np.asarray(idx) // nb)
    amax = bins * nb + k_row.reshape(nbins, nb)[bins].argmax(axis=1)
    pts = np.unique(np.concatenate([np.asarray(idx, dtype=np.int64), amax.astype(np.int64)]))
    ko = np.asarray(oracle_at(pts))
    got = k_row[pts]
    b_of = pts // nb
    bmax = {int(b): float(ko[b_of == b].max()) for b in bins}
    thr = np.array([floor * bmax[int(b)] for b in b_of])
    above = (ko > thr) & (ko > 0)
    assert above.sum() > 0, what
    err = np.abs(got - ko)
    rel = err[above] / ko[above]
    worst = float(rel.max())
    assert worst <= rtol, "%s: max rel err %.3e > %.1e at grid index %d" % (
        what, worst, rtol, int(pts[above][rel.argmax()]))
    below = ~above
    assert np.all(err[below] <= rtol * thr[below]), "%s: error below the floor" % what
    # the device argmax of every touched bin is among the points held to rtol
    # (or the bin is zero on both sides)
    amax_pos = np.searchsorted(pts, amax)
    assert np.all(above[amax_pos] | ((ko[amax_pos] == 0) & (got[amax_pos] == 0))), what
    return worst
