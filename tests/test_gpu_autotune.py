"""The Voigt tile-shape autotuner: it picks one of the built shapes, and the
shape changes no FP64 result (every grid point sums its lines in list order
whatever the tiling) and FP32 results only at rounding level."""
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


def test_autotune_keeps_results(ctx):
    from paper_1503_03806_gb300 import helk
    lines = synth.random_lines(3000, 301, 0.0, 1000.0)
    case = Case(1500.0, 1.0, 18.0, (0.0, 0.01, 100_000 + 17), ("abs", 20.0))
    ctx.upload(lines)
    k64 = case.gpu(ctx).cpu().numpy()
    k32 = case.gpu(ctx, precision=helk.HELK_PREC_F32_KAHAN).cpu().numpy()
    t64 = ctx.autotune(case.T, case.P, case.mass, case.cut, case.grid, precision=helk.HELK_PREC_F64)
    t32 = ctx.autotune(case.T, case.P, case.mass, case.cut, case.grid,
                       precision=helk.HELK_PREC_F32_KAHAN)
    assert t64 in (1024, 1536, 2048) and t32 in (2048, 3072, 4096)
    k64b = case.gpu(ctx).cpu().numpy()
    k32b = case.gpu(ctx, precision=helk.HELK_PREC_F32_KAHAN).cpu().numpy()
    assert np.array_equal(k64, k64b)
    nz = k32 > 0
    assert np.array_equal(nz, k32b > 0)
    assert np.max(np.abs(k32b[nz] - k32[nz]) / k32[nz]) < 2e-6
