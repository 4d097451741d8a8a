"""The Voigt kernel shapes and their autotuner: every candidate shape (tile
width, warps per CTA, candidate lines per pipeline stage) gives the same
FP64 result bit for bit (every grid point sums its lines in list order
whatever the tiling) and the same FP32 result up to rounding; the autotuner
picks one of the candidates and keeps the results."""
import numpy as np
import pytest

from paper_1503_03806_gb300 import synth
from tests.helpers import Case

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


def _case():
    lines = synth.random_lines(3000, 301, 0.0, 1000.0)
    # a grid that is no multiple of any tile: ragged last tile for every shape
    return lines, Case(1500.0, 1.0, 18.0, (0.0, 0.01, 100_000 + 17), ("abs", 20.0))


def test_every_tile_shape_agrees(ctx):
    from paper_1503_03806_gb300 import helk
    lines, case = _case()
    ctx.upload(lines)
    n = case.grid[2]
    for prec in (helk.HELK_PREC_F64, helk.HELK_PREC_F32_KAHAN):
        shapes = helk.helk_tile_candidates(prec)
        assert len(shapes) >= 3
        ref = None
        for t in shapes:
            ctx.set_tile(prec, n, t)
            k = case.gpu(ctx, precision=prec).cpu().numpy()
            if ref is None:
                ref = k
            elif prec == helk.HELK_PREC_F64:
                assert np.array_equal(k, ref), t
            else:
                nz = ref > 0
                assert np.array_equal(nz, k > 0), t
                assert np.max(np.abs(k[nz] - ref[nz]) / ref[nz]) < 2e-6, t
        ctx.set_tile(prec, n, 0)
    with pytest.raises(helk.HelkError):
        ctx.set_tile(helk.HELK_PREC_F32_KAHAN, n, 1000)


def test_autotune_keeps_results(ctx):
    from paper_1503_03806_gb300 import helk
    lines, case = _case()
    ctx.upload(lines)
    k64 = case.gpu(ctx).cpu().numpy()
    k32 = case.gpu(ctx, precision=helk.HELK_PREC_F32_KAHAN).cpu().numpy()
    t64 = ctx.autotune(case.T, case.P, case.mass, case.cut, case.grid, precision=helk.HELK_PREC_F64)
    t32 = ctx.autotune(case.T, case.P, case.mass, case.cut, case.grid,
                       precision=helk.HELK_PREC_F32_KAHAN)
    assert t64 in helk.helk_tile_candidates(helk.HELK_PREC_F64)
    assert t32 in helk.helk_tile_candidates(helk.HELK_PREC_F32_KAHAN)
    k64b = case.gpu(ctx).cpu().numpy()
    k32b = case.gpu(ctx, precision=helk.HELK_PREC_F32_KAHAN).cpu().numpy()
    assert np.array_equal(k64, k64b)
    nz = k32 > 0
    assert np.array_equal(nz, k32b > 0)
    assert np.max(np.abs(k32b[nz] - k32[nz]) / k32[nz]) < 2e-6
