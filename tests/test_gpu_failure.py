"""Failure detection without a GPU fault: a kernel's bounded wait on a
barrier that nothing completes gives up, the host reads HELK_ERR_TIMEOUT at
the next synchronisation, and the context keeps working afterwards."""
import numpy as np
import pytest

from paper_1503_03806_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_03806_gb300 import build
    build.build()
    from paper_1503_03806_gb300 import helk
    ctx = helk.Context(0)
    try:
        assert helk.lib.helk_selftest_timeout(ctx.h, 1000) == helk.HELK_OK
        with pytest.raises(helk.HelkError) as e:
            ctx.sync()
        assert e.value.status == helk.HELK_ERR_TIMEOUT
        ctx.sync()  # reported once
        lines = synth.random_lines(100, 701, 0.0, 50.0)
        ctx.upload(lines)
        k = ctx.opacity(1500.0, 1.0, 18.0, ("abs", 2.0), (0.0, 0.01, 5000))
        ctx.sync()
        assert np.isfinite(k.cpu().numpy()).all() and k.sum().item() > 0
    finally:
        ctx.close()
