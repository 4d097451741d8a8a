"""Batched conditions (one persistent, graph-captured launch) and
multi-species line lists.

A batch must reproduce, bit for bit, the single-condition calls (each grid
point sums the same lines in the same order in the same kernel), also when
the captured graph is replayed with new condition values; the FP64 batch is
held to the oracle at 1e-9 per condition, with exact evaluation counts per
method.
"""
import numpy as np
import pytest

import oracle
from paper_1503_03806_gb300 import synth
from tests.helpers import NTHREADS, Case, assert_rel

pytestmark = pytest.mark.gpu


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


GRID = (0.0, 0.01, 20000 + 37)
CUT = ("lorentz", 500.0, 8.0)


def conditions(seed, n):
    rng = np.random.default_rng(seed)
    T = rng.uniform(500.0, 3000.0, n)
    P = 10.0 ** rng.uniform(-5.0, 2.0, n)
    q = (296.0 / T) ** 1.5
    return T, P, q


@pytest.mark.parametrize("form", ["f64", "f32"])
def test_batch_equals_single_calls(ctx, form):
    from paper_1503_03806_gb300 import helk
    prec = helk.HELK_PREC_F64 if form == "f64" else helk.HELK_PREC_F32_KAHAN
    lines = synth.random_lines(2500, 401, 0.0, 200.0, with_elower=True, strengths="lognormal")
    ctx.upload(lines)
    for seed in (1, 2):  # second pass replays the captured graph with new conditions
        T, P, q = conditions(seed, 7)
        kb = ctx.opacity_batch(T, P, 18.0, CUT, GRID, precision=prec, q_ratio=q).cpu().numpy()
        for k in range(7):
            ks = ctx.opacity(T[k], P[k], 18.0, CUT, GRID, precision=prec, q_ratio=q[k]).cpu().numpy()
            assert np.array_equal(kb[k], ks), (seed, k)


def test_batch_fp64_against_oracle_with_counts(ctx):
    lines = synth.random_lines(1500, 402, 0.0, 200.0, with_elower=True, strengths="lognormal",
                               extra_fields=True)
    ctx.upload(lines)
    T, P, q = conditions(3, 5)
    kb = ctx.opacity_batch(T, P, 18.0, CUT, GRID, q_ratio=q, count_regions=True).cpu().numpy()
    ev, reg = ctx.batch_stats(5, with_regions=True)
    for k in range(5):
        case = Case(T[k], P[k], 18.0, GRID, CUT, q_ratio=q[k])
        ko, evo, rego = oracle.opacity(lines, case.oracle_cond(), nthreads=NTHREADS)
        assert ev[k] == evo and np.array_equal(reg[k, :3], rego), k
        assert_rel(kb[k], ko, 1e-9, "condition %d" % k)


def test_batch_kdist_of_all_conditions(ctx):
    # one helk_kdist call over the batch output (n_cond x nbins bins) against
    # the oracle's opacity and tables of each condition
    lines = synth.random_lines(1000, 403, 0.0, 200.0)
    ctx.upload(lines)
    T, P, q = conditions(4, 4)
    grid = (0.0, 0.01, 20000)
    kb = ctx.opacity_batch(T, P, 18.0, ("abs", 5.0), grid)
    coef, mean, srt = ctx.kdist(kb.view(-1), 4 * 10, 12, want_sorted=True)
    for k in range(4):
        ko, _, _ = oracle.opacity(lines, Case(T[k], P[k], 18.0, grid, ("abs", 5.0)).oracle_cond(),
                                  nthreads=NTHREADS)
        s_or, c_or, m_or = oracle.kdist(ko, 10, 12)
        assert_rel(srt.view(4, -1)[k].cpu().numpy(), s_or, 1e-9, "sorted, condition %d" % k)
        c = coef.view(4, 10, 12)[k].cpu().numpy()
        assert np.max(np.abs(c - c_or) / np.max(np.abs(c_or), axis=1, keepdims=True)) < 1e-9


def test_mixed_species_list(ctx):
    # two species in one list: per-line mass and abundance weight (Sec. 2.1)
    A = synth.random_lines(800, 404, 0.0, 200.0)
    B = synth.random_lines(700, 405, 0.0, 200.0)
    mix = {k: np.concatenate([A[k], B[k]]) for k in A}
    mix["mass"] = np.concatenate([np.full(800, 18.0), np.full(700, 44.0)])
    mix["weight"] = np.concatenate([np.full(800, 0.8), np.full(700, 0.2)])
    order = np.argsort(mix["nu0"], kind="stable")
    mix = {k: v[order] for k, v in mix.items()}
    case = Case(1300.0, 0.7, 18.0, GRID, ("abs", 6.0))
    ctx.upload(mix)
    k = case.gpu(ctx, count_regions=True).cpu().numpy()
    ev, reg = ctx.stats(with_regions=True)
    ko, evo, rego = oracle.opacity(mix, case.oracle_cond(), nthreads=NTHREADS)
    assert ev == evo and np.array_equal(reg[:3], rego)
    assert_rel(k, ko, 1e-9, "mixed species")


@pytest.mark.parametrize("form", ["f64", "f32"])
def test_chunked_batch_equals_one_chunk(ctx, form):
    # a record budget of three conditions' records runs 8 conditions as
    # chunks of 3, 3 and 2 (each its own graph): the same results bit for bit
    # and the same per-condition statistics as one chunk, also on a replay
    from paper_1503_03806_gb300 import helk
    prec = helk.HELK_PREC_F64 if form == "f64" else helk.HELK_PREC_F32_KAHAN
    lines = synth.random_lines(2000, 406, 0.0, 200.0, with_elower=True, strengths="lognormal")
    ctx.upload(lines)
    T, P, q = conditions(5, 8)
    k1 = ctx.opacity_batch(T, P, 18.0, CUT, GRID, precision=prec, q_ratio=q, count_regions=True).cpu().numpy()
    ev1, reg1 = ctx.batch_stats(8, with_regions=True)
    per_line = 64 if form == "f64" else 120
    try:
        ctx.set_batch_budget(3 * 2000 * per_line)
        for _ in range(2):
            k3 = ctx.opacity_batch(T, P, 18.0, CUT, GRID, precision=prec, q_ratio=q,
                                   count_regions=True).cpu().numpy()
            ev3, reg3 = ctx.batch_stats(8, with_regions=True)
            assert np.array_equal(k1, k3)
            assert np.array_equal(ev1, ev3) and np.array_equal(reg1, reg3)
        # one condition a chunk, without counting (the counting variant has a
        # kernel shape of its own, whose FP32 sums group differently)
        ctx.set_batch_budget(0)
        k1n = ctx.opacity_batch(T, P, 18.0, CUT, GRID, precision=prec, q_ratio=q).cpu().numpy()
        ctx.set_batch_budget(1)
        k8 = ctx.opacity_batch(T, P, 18.0, CUT, GRID, precision=prec, q_ratio=q).cpu().numpy()
        assert np.array_equal(k1n, k8)
    finally:
        ctx.set_batch_budget(0)
