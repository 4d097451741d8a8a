"""The library on a caller's stream: every call of a context is ordered on
the stream it was given, including the FP32 form's Algorithm 916 cores,
which run on the context's own second stream beside the main Voigt kernel
and join back before their sums are added.  Synchronising the caller's
stream alone must therefore see complete results, equal bit for bit to
those on the default stream, and work queued on the caller's stream before
a call must be complete when the call starts."""
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
    # low pressure, fine grid, short cutoff: most evaluations are Algorithm 916
    # cores, so the core kernel on the second stream outlasts the main kernel
    lines = synth.random_lines(3000, 17, 10000.0, 10300.0)
    return lines, Case(1500.0, 0.01, 18.0, (10000.0, 0.001, 300_000 + 3), ("abs", 0.3))


def test_results_on_a_caller_stream_equal_the_default_stream(ctx):
    import torch
    from paper_1503_03806_gb300 import helk
    lines, case = _case()
    ctx.upload(lines)
    n = case.grid[2]
    ref = case.gpu(ctx, precision=helk.HELK_PREC_F32_KAHAN).cpu().numpy()
    coef_ref, mean_ref, _ = ctx.kdist(torch.from_numpy(ref).cuda(), 1, 20)
    coef_ref, mean_ref = coef_ref.cpu().numpy(), mean_ref.cpu().numpy()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    ctx.set_stream(s)
    try:
        with torch.cuda.stream(s):
            out = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
            for _ in range(3):
                k = case.gpu(ctx, out=out, precision=helk.HELK_PREC_F32_KAHAN)
                coef, mean, _ = ctx.kdist(k, 1, 20)
        s.synchronize()  # the caller's stream only
        assert np.array_equal(out.cpu().numpy(), ref)
        assert np.array_equal(coef.cpu().numpy(), coef_ref)
        assert np.array_equal(mean.cpu().numpy(), mean_ref)
        # work queued before the call on the caller's stream comes first
        ref_t = torch.from_numpy(ref).cuda()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            out.copy_(ref_t)
            case.gpu(ctx, out=out, precision=helk.HELK_PREC_F32_KAHAN, accumulate=True)
        s.synchronize()
        got = out.cpu().numpy()
        nz = ref > 0
        assert nz.sum() > 0.5 * n
        assert np.max(np.abs(got[nz] - 2.0 * ref[nz]) / (2.0 * ref[nz])) < 1e-13
    finally:
        ctx.set_stream(None)
        torch.cuda.synchronize()
