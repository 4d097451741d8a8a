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
  point grid at 0.001 cm^-1: all 16 conditions in one FP32 batch call, then
  the k-tables of all of them (16000 bins of 30000 points) in one call;
  sampled points of five conditions, whole bins of four, and the k-tables of
  those bins (on the oracle's opacity) against the oracle.
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


def mixed_lines(w):
    """The 4-species list of the mixed workload (2.5e7 lines each, masses 18,
    16, 44, 17 amu, mixing ratio 1/4 each) as one list with per-line mass and
    abundance weight, ordered by nu0."""
    parts = []
    for s, (m, x) in enumerate(zip(w["species_mass"], w["mixing"])):
        L = synth.workload_lines("mixed", species=s)
        L["mass"] = np.full(L["nu0"].shape[0], m)
        L["weight"] = np.full(L["nu0"].shape[0], x)
        parts.append(L)
    lines = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    del parts
    order = np.argsort(lines["nu0"], kind="stable")
    return {k: np.ascontiguousarray(v[order]) for k, v in lines.items()}


def test_mixed_batch_full_size(ctx):
    # The mixed workload as specified: 1e8 lines of 4 species, all 4 T x 4 P
    # conditions in one helk_opacity_batch call (FP32 form; its records, 120 B
    # a line and condition, run in chunks under the 64 GiB record budget) on
    # the 3e7-point grid, then the k-tables of all 16 conditions (16000 bins
    # of 30000 points, 20 coefficients) in one helk_kdist call.
    import torch
    from paper_1503_03806_gb300 import helk
    w = synth.WORKLOADS["mixed"]
    lines = mixed_lines(w)
    grid = (w["nu_min"], w["dnu"], w["ngrid"])
    Ts = np.repeat(np.asarray(w["T"]), len(w["P_atm"]))
    Ps = np.tile(np.asarray(w["P_atm"]), len(w["T"]))
    qs = (296.0 / Ts) ** 1.5
    nb = grid[2] // w["nbins"]
    ctx.upload(lines)
    kb = ctx.opacity_batch(Ts, Ps, 18.0, w["cut"], grid, precision=helk.HELK_PREC_F32_KAHAN, q_ratio=qs)
    ev, _ = ctx.batch_stats(len(Ts))
    assert np.all(ev > 0)
    reach = w["cut"][2] + grid[1]
    rng = np.random.default_rng(5)

    def oracle_at(cond):
        def at(pts):
            near = near_lines(lines, grid[0] + pts[0] * grid[1], grid[0] + pts[-1] * grid[1], reach)
            return oracle.opacity_points(near, cond, pts)[0]
        return at

    # sampled points of five conditions (cold and hot, every pressure), two
    # regions of 30 points each, against the oracle
    for c in (0, 5, 10, 15, 3):
        cond = Case(Ts[c], Ps[c], 18.0, grid, w["cut"], q_ratio=qs[c]).oracle_cond()
        row = kb[c].cpu().numpy()
        assert np.all(np.isfinite(row)) and row.max() > 0
        for lo in (3000.0, 21000.0):
            i0 = int((lo - grid[0]) / grid[1])
            idx = np.sort(rng.choice(np.arange(i0, i0 + 100_000), 30, replace=False))
            check_sampled_f32(row, w["nbins"], idx, oracle_at(cond), RTOL32, FLOOR,
                              "mixed condition %d at %g" % (c, lo))
        del row
    # whole bins from the oracle at the two low pressures (cheap there):
    # the device's opacity of those bins, then the k-tables of the full
    # 16-condition array with those bins replaced by the oracle's opacity,
    # against the oracle's own tables (sorted values bit for bit)
    checks = []
    for c in (0, 1, 12, 13):
        cond = Case(Ts[c], Ps[c], 18.0, grid, w["cut"], q_ratio=qs[c]).oracle_cond()
        for b in (17, 611):
            pts = np.arange(b * nb, (b + 1) * nb)
            ko = oracle_at(cond)(pts)
            got = kb[c, b * nb:(b + 1) * nb].cpu().numpy()
            thr = FLOOR * ko.max()
            sel = ko > thr
            if sel.any():
                err = np.abs(got[sel] - ko[sel]) / ko[sel]
                assert err.max() <= RTOL32, ("whole bin", c, b, float(err.max()))
            assert np.all(np.abs(got[~sel] - ko[~sel]) <= RTOL32 * max(thr, 0.0)), ("below floor", c, b)
            checks.append((c * w["nbins"] + b, ko))
    kk = kb.view(-1)
    for gb, ko in checks:
        kk[gb * nb:(gb + 1) * nb] = torch.from_numpy(ko).cuda()
    coef, mean, srt = ctx.kdist(kk, len(Ts) * w["nbins"], w["ncheb"], want_sorted=True)
    for gb, ko in checks:
        s_or, c_or, m_or = oracle.kdist(ko, 1, w["ncheb"])
        assert np.array_equal(srt[gb * nb:(gb + 1) * nb].cpu().numpy(), s_or), gb
        c = coef[gb].cpu().numpy()
        assert np.max(np.abs(c - c_or[0])) <= 1e-9 * np.max(np.abs(c_or[0])), gb
        assert abs(float(mean[gb]) - m_or[0]) <= 1e-12 * abs(m_or[0]) or m_or[0] == float(mean[gb]), gb
    # every other bin: the sorted output is a non-decreasing permutation of
    # its input (checked on a sample of bins at full size)
    for gb in rng.choice(len(Ts) * w["nbins"], 6, replace=False):
        a = kk[gb * nb:(gb + 1) * nb].cpu().numpy()
        assert np.array_equal(srt[gb * nb:(gb + 1) * nb].cpu().numpy(), np.sort(a)), gb
    del kb, kk, srt, lines
    torch.cuda.empty_cache()
