"""Parity at the full sizes of the larger workloads, in the launch
configurations the benchmark times, on sampled grid points the oracle
computes one by one.

- tp_grid: 1e6 lines (log-normal strengths, lower-state energies), all
  8 T x 8 P conditions in one graph-captured FP32 batch with an autotuned
  tile, and an FP64 batch of 8 of them; sampled points of several
  conditions against the oracle (FP64: 1e-9; FP32: 1e-5 where kappa exceeds
  1e-8 of its bin maximum).
- mixed: 4 species x 2.5e7 lines (masses 18, 16, 44, 17 amu, mixing 1/4
  each) in one upload with per-line mass and abundance weight, on the 3e7
  point grid at 0.001 cm^-1; one condition in the FP32 form.
- the largest grid accepted (2^31 - 4097 points), both forms: lines at both
  ends and beyond index 2^30, and, without a cutoff, lines whose centres lie
  outside the int32 range of grid indices.

The oracle sums every line of the list whose window holds the point.  For
the 1e8-line list it is given, per sampled region, the lines whose centre
lies within the largest possible window half-width (the 100 cm^-1 cap plus
a grid step) of the region: no other line can reach those points, so its
sums are the full list's.  The FP32 checks take every threshold from the
oracle: each touched bin's floor is 1e-8 of the largest oracle value among
its checked points, and those include the device's largest point of the
bin, itself held to 1e-5, so a device value inflated anywhere in a touched
bin fails (tests/helpers.py: check_sampled_f32).
"""
import numpy as np
import pytest

import oracle
from paper_1503_03806_gb300 import synth
from tests.helpers import Case, assert_rel, check_sampled_f32, near_lines

pytestmark = pytest.mark.gpu

RTOL64 = 1e-9
RTOL32 = 1e-5
FLOOR = 1e-8


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_03806_gb300 import build
    build.build()
    from paper_1503_03806_gb300 import helk
    c = helk.Context(0)
    yield c
    c.close()


def _sample_idx(ngrid, seed, n=120):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.integers(0, ngrid, n), [0, ngrid - 1]]))


def test_tp_grid_batches(ctx):
    import torch
    from paper_1503_03806_gb300 import helk
    w = synth.WORKLOADS["tp_grid"]
    lines = synth.workload_lines("tp_grid")
    Ts = np.repeat(np.asarray(w["T"]), len(w["P_atm"]))
    Ps = np.tile(np.asarray(w["P_atm"]), len(w["T"]))
    qs = (296.0 / Ts) ** 1.5
    grid = (w["nu_min"], w["dnu"], w["ngrid"])
    ctx.upload(lines)
    ctx.autotune(Ts[0], Ps[-1], w["mass"], w["cut"], grid, precision=helk.HELK_PREC_F32_KAHAN, q_ratio=qs[0])
    kb = torch.empty((len(Ts), grid[2]), dtype=torch.float64, device="cuda")
    ctx.opacity_batch(Ts, Ps, w["mass"], w["cut"], grid, out=kb, precision=helk.HELK_PREC_F32_KAHAN,
                      q_ratio=qs)
    ctx.opacity_batch(Ts, Ps, w["mass"], w["cut"], grid, out=kb, precision=helk.HELK_PREC_F32_KAHAN,
                      q_ratio=qs)  # a replay of the captured graph
    k32 = kb.cpu().numpy()
    sub = np.array([0, 9, 27, 36, 54, 63])  # cold/hot x low/high pressure
    k64 = ctx.opacity_batch(Ts[sub], Ps[sub], w["mass"], w["cut"], grid, precision=helk.HELK_PREC_F64,
                            q_ratio=qs[sub]).cpu().numpy()
    idx = _sample_idx(grid[2], 31)
    for j, c in enumerate(sub):
        case = Case(Ts[c], Ps[c], w["mass"], grid, w["cut"], q_ratio=qs[c])
        ko, _ = oracle.opacity_points(lines, case.oracle_cond(), idx)
        assert_rel(k64[j][idx], ko, RTOL64, "tp_grid FP64 condition %d" % c)
        cond = case.oracle_cond()
        check_sampled_f32(k32[c], w["nbins"], idx, lambda pts: oracle.opacity_points(lines, cond, pts)[0],
                          RTOL32, FLOOR, "tp_grid FP32 condition %d" % c)


NMAX = 2**31 - 1 - 4096  # the largest grid the library accepts


def _region_idx(centres, halfwidth, n):
    idx = np.concatenate([np.arange(max(0, c - halfwidth), min(n, c + halfwidth + 1)) for c in centres])
    return np.unique(idx)


def _check_points(k_dev, idx, ko, rtol, floor, what):
    """Compare the device result at idx (a gather on the device) with the
    oracle: every point for rtol 1e-9, else points above floor x max."""
    import torch
    got = k_dev[torch.from_numpy(idx).cuda()].cpu().numpy()
    sel = (ko > floor * ko.max()) & (ko > 0) if floor else ko != 0
    assert sel.sum() > 0, what
    err = np.abs(got[sel] - ko[sel]) / ko[sel]
    assert err.max() <= rtol, (what, float(err.max()))
    assert np.all(got[ko == 0] == 0.0), what


def test_largest_grid(ctx):
    # 2^31 - 4097 points (the largest grid accepted): line centres near both
    # ends and at index ~1.5e9, windows of 50 points (Algorithm 916 cores near
    # the end, where the Doppler width is large; GH1 wings near the start);
    # then, without a cutoff, lines whose centres lie far outside the grid on
    # both sides (beyond the int32 range of grid indices) reach every point
    import torch
    from paper_1503_03806_gb300 import helk
    n, dnu = NMAX, 0.001
    rng = np.random.default_rng(77)
    end = (n - 1) * dnu
    nu = np.sort(np.concatenate([rng.uniform(0.02, 0.06, 6), rng.uniform(1.5e6, 1.5e6 + 0.04, 6),
                                 rng.uniform(end - 0.05, end + 0.01, 6)]))
    lines = {"nu0": nu, "S0": 10.0 ** rng.uniform(-24, -20, nu.size), "gamma_air": rng.uniform(0.02, 0.1, nu.size)}
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    case = Case(1500.0, 1.0, 18.0, (0.0, dnu, n), ("abs", 0.05))
    ctx.upload(lines)
    cidx = np.rint(nu / dnu).astype(np.int64)
    idx = _region_idx(cidx, 80, n)
    ko, evo = oracle.opacity_points(lines, case.oracle_cond(), idx)
    case.gpu(ctx, out=out, count_regions=True)
    ev, reg = ctx.stats(with_regions=True)
    _check_points(out, idx, ko, 1e-9, 0.0, "largest grid FP64")
    assert reg[0] > 0 and reg[2] > 0  # Algorithm 916 and GH1 both used
    case.gpu(ctx, out=out, precision=helk.HELK_PREC_F32_KAHAN)
    _check_points(out, idx, ko, 1e-5, 1e-8, "largest grid FP32")
    assert float(out[-1]) > 0.0 and float(out[0]) > 0.0
    # no cutoff: two lines inside, two far outside (grid starts at 3e6 cm^-1)
    nu2 = np.array([10.0, 3.0e6 + 0.03, 3.0e6 + end - 0.02, 9.0e6])
    lines2 = {"nu0": nu2, "S0": np.array([1e-20, 1e-22, 1e-22, 1e-20]),
              "gamma_air": np.array([0.05, 0.07, 0.03, 0.08])}
    case2 = Case(1500.0, 1.0, 18.0, (3.0e6, dnu, n), ("none",))
    ctx.upload(lines2)
    idx2 = np.unique(np.concatenate([_region_idx([30, n - 20], 60, n),
                                     rng.integers(0, n, 200), [0, n - 1]]))
    ko2, _ = oracle.opacity_points(lines2, case2.oracle_cond(), idx2)
    case2.gpu(ctx, out=out)
    _check_points(out, idx2, ko2, 1e-9, 0.0, "largest grid, no cutoff, FP64")
    case2.gpu(ctx, out=out, precision=helk.HELK_PREC_F32_KAHAN)
    _check_points(out, idx2, ko2, 1e-5, 1e-8, "largest grid, no cutoff, FP32")
    del out
    torch.cuda.empty_cache()


def test_mixed_species_full_size(ctx):
    import torch
    from paper_1503_03806_gb300 import helk
    w = synth.WORKLOADS["mixed"]
    parts = []
    for s, (m, x) in enumerate(zip(w["species_mass"], w["mixing"])):
        L = synth.workload_lines("mixed", species=s)
        L["mass"] = np.full(L["nu0"].shape[0], m)
        L["weight"] = np.full(L["nu0"].shape[0], x)
        parts.append(L)
    lines = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    del parts
    order = np.argsort(lines["nu0"], kind="stable")
    lines = {k: np.ascontiguousarray(v[order]) for k, v in lines.items()}
    del order
    grid = (w["nu_min"], w["dnu"], w["ngrid"])
    T, P = w["T"][2], w["P_atm"][2]
    case = Case(T, P, 18.0, grid, w["cut"], q_ratio=(296.0 / T) ** 1.5)
    ctx.upload(lines)
    k = case.gpu(ctx, precision=helk.HELK_PREC_F32_KAHAN).cpu().numpy()
    assert np.all(np.isfinite(k)) and k.max() > 0
    # three regions of 40 points; the oracle gets every line that can reach them
    rng = np.random.default_rng(5)
    reach = w["cut"][2] + grid[1]
    cond = case.oracle_cond()

    def oracle_at(pts):
        near = near_lines(lines, grid[0] + pts[0] * grid[1], grid[0] + pts[-1] * grid[1], reach)
        return oracle.opacity_points(near, cond, pts)[0]

    for lo in (1000.0, 14000.0, 29000.0):
        i0 = int((lo - grid[0]) / grid[1])
        idx = np.sort(rng.choice(np.arange(i0, i0 + 200_000), 40, replace=False))
        check_sampled_f32(k, w["nbins"], idx, oracle_at, RTOL32, FLOOR, "mixed FP32 at %g" % lo)
    del lines
    torch.cuda.empty_cache()
