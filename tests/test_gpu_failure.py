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


def test_oversized_request_reports_oom_and_context_survives():
    # 160 conditions of a 2^31 - 4097-point grid into the library's own
    # opacity buffer: 2.75 TB, beyond any device.  The buffer's cudaMalloc
    # fails (an ordinary error return, no GPU fault), the call returns
    # HELK_ERR_OOM with its message, and the same context then runs a
    # normal call.
    import ctypes
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_03806_gb300 import build
    build.build()
    from paper_1503_03806_gb300 import helk
    ctx = helk.Context(0)
    try:
        ctx.upload(synth.random_lines(50, 702, 10.0, 20.0))
        n_cond, n = 160, 2 ** 31 - 4097
        T = np.full(n_cond, 1500.0)
        P = np.full(n_cond, 1.0)
        g = helk.helk_grid(0.0, 0.01, n)
        o = helk.helk_opts(helk.HELK_PREC_F32_KAHAN, 0, 1.0, 1.0, 0, 0)
        st = helk.lib.helk_opacity_batch(ctx.h, n_cond, T.ctypes.data_as(helk._P), P.ctypes.data_as(helk._P),
                                         None, 18.0, ctypes.byref(helk._cut(("abs", 1.0))), ctypes.byref(g),
                                         ctypes.byref(o), None)
        assert st == helk.HELK_ERR_OOM, st
        assert "out of device memory" in helk.helk_last_error(ctx.h)
        ctx.sync()
        k = ctx.opacity(1500.0, 1.0, 18.0, ("abs", 2.0), (10.0, 0.01, 1000),
                        precision=helk.HELK_PREC_F32_KAHAN)
        ctx.sync()
        assert np.isfinite(k.cpu().numpy()).all() and k.sum().item() > 0
    finally:
        ctx.close()
