"""GPU parity of the opacity stage (Sec. 2.3-2.4): the CUDA path through the
C ABI against the FP64 oracle on the same seeded inputs.

FP64 form: 1e-9 relative per grid point (every term is computed from the
same correctly rounded line parameters; what differs is FMA contraction,
division and libm-vs-CUDA exp/erfcx/sincos rounding, ~1e-15).  Window
bounds and the method chosen for each evaluation depend only on correctly
rounded operations, so evaluation counts per method must match exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1503_03806_gb300 import synth
from tests.helpers import NTHREADS, Case, assert_rel, workload_case

pytestmark = pytest.mark.gpu

RTOL64 = 1e-9


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


def run_both(ctx, lines, case, count=True, **kw):
    ctx.upload(lines)
    k = case.gpu(ctx, count_regions=count, **kw)
    ev, reg = ctx.stats(with_regions=count)
    ko, evo, rego = oracle.opacity(lines, case.oracle_cond(), nthreads=NTHREADS)
    return k.cpu().numpy(), ev, reg, ko, evo, rego


@pytest.mark.parametrize("ngrid", [2048, 20000 + 123, 1])
def test_random_lines_abs_cutoff(ctx, ngrid):
    lines = synth.random_lines(500, 101, 0.05, 201.0)
    case = Case(1500.0, 1.0, 18.0, (0.0, 0.01, ngrid), ("abs", 3.0))
    k, ev, reg, ko, evo, rego = run_both(ctx, lines, case)
    assert ev == evo
    assert np.array_equal(reg[:3], rego)
    assert_rel(k, ko, RTOL64, "abs cutoff")


def test_lorentz_cutoff_all_fields(ctx):
    lines = synth.random_lines(800, 102, 0.0, 300.0, with_elower=True, strengths="lognormal",
                               extra_fields=True)
    case = Case(2300.0, 3.7, 44.0, (1.0, 0.01, 29000 + 7), ("lorentz", 500.0, 12.0), q_ratio=0.31)
    k, ev, reg, ko, evo, rego = run_both(ctx, lines, case)
    assert ev == evo and np.array_equal(reg[:3], rego)
    assert_rel(k, ko, RTOL64, "lorentz cutoff")


def test_no_cutoff_full_profile(ctx):
    lines = synth.random_lines(40, 103, 1000.0, 1030.0)
    case = Case(900.0, 0.2, 16.0, (1000.0, 0.005, 6000 + 11), ("none",))
    k, ev, reg, ko, evo, rego = run_both(ctx, lines, case)
    assert ev == evo == 40 * 6011 and np.array_equal(reg[:3], rego)
    assert rego[0] > 0 and rego[1] > 0 and rego[2] > 0
    assert_rel(k, ko, RTOL64, "no cutoff")


@pytest.mark.parametrize("P", [1e-7, 1e-2, 100.0])
def test_pressure_extremes(ctx, P):
    # tiny P: core region everywhere, windows of 0-1 points; large P: wings
    lines = synth.random_lines(300, 104, 0.0, 100.0, with_elower=True)
    case = Case(3000.0, P, 18.0, (0.0, 0.01, 10000), ("lorentz", 500.0, 100.0), q_ratio=0.2)
    k, ev, reg, ko, evo, rego = run_both(ctx, lines, case)
    assert ev == evo and np.array_equal(reg[:3], rego)
    assert_rel(k, ko, RTOL64, "P=%g" % P)


def test_zero_pressure_gaussian_limit(ctx):
    lines = synth.random_lines(50, 105, 10.0, 20.0)
    case = Case(1500.0, 0.0, 18.0, (10.0, 0.001, 10000), ("abs", 0.5))
    k, ev, reg, ko, evo, rego = run_both(ctx, lines, case)
    assert ev == evo and np.array_equal(reg[:3], rego)
    assert_rel(k, ko, RTOL64, "P=0")


def test_empty_line_list_and_outside_grid(ctx):
    import torch
    empty = {k: np.zeros(0) for k in ("nu0", "S0", "gamma_air")}
    ctx.upload(empty)
    k = ctx.opacity(1500.0, 1.0, 18.0, ("abs", 25.0), (0.0, 0.01, 5000))
    assert torch.count_nonzero(k).item() == 0
    far = {"nu0": np.array([5000.0, 6000.0]), "S0": np.array([1e-20, 1e-20]),
           "gamma_air": np.array([0.05, 0.05])}
    ctx.upload(far)
    k = ctx.opacity(1500.0, 1.0, 18.0, ("abs", 25.0), (0.0, 0.01, 5000), count_regions=True)
    ev, reg = ctx.stats(with_regions=True)
    assert ev == 0 and reg.sum() == 0 and torch.count_nonzero(k).item() == 0


def test_unsorted_upload_gives_same_result(ctx):
    lines = synth.random_lines(700, 106, 0.0, 150.0, extra_fields=True)
    case = Case(1200.0, 2.0, 18.0, (0.0, 0.01, 15000), ("abs", 4.0))
    ctx.upload(lines)
    k_sorted = case.gpu(ctx).cpu().numpy()
    perm = np.random.default_rng(0).permutation(700)
    ctx.upload({k: v[perm] for k, v in lines.items()})
    k_shuf = case.gpu(ctx).cpu().numpy()
    assert np.array_equal(k_sorted, k_shuf)


def test_device_side_upload_and_accumulate(ctx):
    import torch
    lines = synth.random_lines(400, 107, 0.0, 100.0)
    case = Case(1500.0, 1.0, 18.0, (0.0, 0.01, 10000), ("abs", 5.0))
    dev = {k: torch.from_numpy(v).cuda() for k, v in lines.items()}
    A = {k: v[::2] for k, v in dev.items()}
    B = {k: v[1::2] for k, v in dev.items()}
    ctx.upload(A)
    out = case.gpu(ctx, weight=0.7)
    ctx.upload(B)
    out = case.gpu(ctx, out=out, accumulate=True, weight=0.3)
    la = {k: v[::2] for k, v in lines.items()}
    lb = {k: v[1::2] for k, v in lines.items()}
    ka, _, _ = oracle.opacity(la, case.oracle_cond(), weight=0.7)
    kab, _, _ = oracle.opacity(lb, case.oracle_cond(), weight=0.3, kappa=ka)
    assert_rel(out.cpu().numpy(), kab, RTOL64, "accumulate")


def test_small_workload_full_grid(ctx):
    # 1e4 lines, 3e5 points, cutoff 25 cm^-1: the whole grid against the oracle
    w = synth.WORKLOADS["small"]
    lines = synth.workload_lines("small")
    case = workload_case(w)
    k, ev, reg, ko, evo, rego = run_both(ctx, lines, case)
    assert ev == evo and np.array_equal(reg[:3], rego)
    assert_rel(k, ko, RTOL64, "small workload")


def test_medium_workload_sampled_points(ctx):
    # 1e5 lines, 3e6 points, cutoff 100 cm^-1 at full size, in the launch
    # configuration of the benchmark; the oracle computes sampled points.
    w = synth.WORKLOADS["medium"]
    lines = synth.workload_lines("medium")
    case = workload_case(w)
    ctx.upload(lines)
    k = case.gpu(ctx).cpu().numpy()
    ev, _ = ctx.stats()
    r = oracle.lineprep(lines, case.oracle_cond())
    assert ev == int(np.maximum(r["ihi"] - r["ilo"] + 1, 0).sum())
    rng = np.random.default_rng(7)
    idx = np.concatenate([rng.integers(0, w["ngrid"], 1500), np.arange(0, 400),
                          np.arange(w["ngrid"] - 400, w["ngrid"]), np.arange(1_500_000, 1_500_600)])
    ko, _ = oracle.opacity_points(lines, case.oracle_cond(), idx)
    assert_rel(k[idx], ko, RTOL64, "medium workload (sampled)")


def test_invalid_arguments(ctx):
    from paper_1503_03806_gb300 import helk
    lines = synth.random_lines(10, 108, 0.0, 10.0)
    ctx.upload(lines)
    bad = [dict(T=-1.0), dict(T=float("nan")), dict(P=-1.0), dict(mass=0.0)]
    for b in bad:
        args = dict(T=1500.0, P=1.0, mass=18.0)
        args.update(b)
        with pytest.raises(helk.HelkError) as e:
            ctx.opacity(args["T"], args["P"], args["mass"], ("abs", 1.0), (0.0, 0.01, 100))
        assert e.value.status == helk.HELK_ERR_INVALID_ARG
    with pytest.raises(helk.HelkError):
        ctx.opacity(1500.0, 1.0, 18.0, ("abs", 1.0), (0.0, -0.01, 100))
    with pytest.raises(helk.HelkError):
        ctx.opacity(1500.0, 1.0, 18.0, ("abs", -1.0), (0.0, 0.01, 100))
    bad_lines = dict(lines)
    bad_lines["S0"] = lines["S0"].copy()
    bad_lines["S0"][3] = -1.0
    with pytest.raises(helk.HelkError) as e:
        ctx.upload(bad_lines)
    assert e.value.status == helk.HELK_ERR_INVALID_ARG
    for badval in (float("inf"), float("nan"), 0.0, -3.0):
        nan_lines = dict(lines)
        nan_lines["nu0"] = lines["nu0"].copy()
        nan_lines["nu0"][0] = badval
        with pytest.raises(helk.HelkError):
            ctx.upload(nan_lines)
