"""Failure detection without a GPU fault: a kernel's bounded wait on a
barrier that nothing completes gives up after its time limit (read from the
GPU's global timer, not counted in polls), the host reads HELK_ERR_TIMEOUT at
the next synchronisation, and the context keeps working afterwards."""
import numpy as np
import pytest

from paper_1503_03806_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit_ms", [5, 40])
def test_bounded_wait_reports_timeout_and_context_survives(limit_ms):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_03806_gb300 import build
    build.build()
    from paper_1503_03806_gb300 import helk
    ctx = helk.Context(0)
    try:
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        assert helk.lib.helk_selftest_timeout(ctx.h, limit_ms * 1000) == helk.HELK_OK
        e1.record()
        with pytest.raises(helk.HelkError) as e:
            ctx.sync()
        assert e.value.status == helk.HELK_ERR_TIMEOUT
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        # the wait lasts its limit, and not much longer (one poll's suspension
        # and the launch)
        assert limit_ms * 0.99 <= ms <= limit_ms + 20.0, ms
        ctx.sync()  # reported once
        lines = synth.random_lines(100, 701, 0.0, 50.0)
        ctx.upload(lines)
        k = ctx.opacity(1500.0, 1.0, 18.0, ("abs", 2.0), (0.0, 0.01, 5000))
        ctx.sync()
        assert np.isfinite(k.cpu().numpy()).all() and k.sum().item() > 0
    finally:
        ctx.close()


def test_selftest_limit_is_checked():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_03806_gb300 import build
    build.build()
    from paper_1503_03806_gb300 import helk
    ctx = helk.Context(0)
    try:
        assert helk.lib.helk_selftest_timeout(ctx.h, 0) == helk.HELK_ERR_INVALID_ARG
        assert helk.lib.helk_selftest_timeout(ctx.h, 10 * 1000 * 1000 + 1) == helk.HELK_ERR_INVALID_ARG
    finally:
        ctx.close()
