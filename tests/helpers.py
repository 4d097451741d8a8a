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
