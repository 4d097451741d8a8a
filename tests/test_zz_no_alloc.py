"""The allocation-free k-distribution entry point, helk_kdist_static, called
through the C ABI, against the regular entry point helk_kdist.

helk_kdist_static serves callers that cannot allocate device memory, such as
code inside a framework whose caching allocator owns the device memory, or a
host program that allows no allocation once its set-up is done: its scratch
is a fixed device array inside the library.  Its outputs must equal those of
helk_kdist within the k-distribution tests' tolerances (sorted values bit for
bit, coefficients to 1e-9 of max|c|, bin means to 1e-12), on consecutive calls
that reuse the scratch, replace its contents with other sizes, and then go
back to the first sizes.  This file is collected last on purpose: it passes
alone in a fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1503_03806_gb300 import synth

pytestmark = pytest.mark.gpu


def _call_static(helk, kappa, nbins, ncheb, floor, stream):
    import torch
    coef = torch.empty((nbins, ncheb), dtype=torch.float64, device="cuda")
    mean = torch.empty(nbins, dtype=torch.float64, device="cuda")
    srt = torch.empty_like(kappa)
    st = helk.lib.helk_kdist_static(ctypes.c_void_p(kappa.data_ptr()), kappa.shape[0], nbins, ncheb,
                                    floor, ctypes.c_void_p(coef.data_ptr()),
                                    ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(srt.data_ptr()),
                                    ctypes.c_void_p(stream))
    return st, coef, mean, srt


def test_static_entry_point_matches_regular():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_03806_gb300 import build
    build.build()
    from paper_1503_03806_gb300 import helk
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = helk.Context(0)
    try:
        # two calls in a row with the same sizes (the second reuses the
        # scratch), one with new sizes (the scratch is rebuilt), then the
        # first sizes again (rebuilt once more)
        for nbins, nb, ncheb, seed in [(30, 10000, 20, 1), (30, 10000, 20, 2), (7, 12288, 32, 3),
                                       (30, 10000, 20, 4)]:
            k = torch.from_numpy(synth.uniform_kappa(nbins * nb, seed)).cuda()
            st, coef, mean, srt = _call_static(helk, k, nbins, ncheb, 1e-250, stream)
            torch.cuda.synchronize()
            assert st == helk.HELK_OK, st
            c_r, m_r, s_r = ctx.kdist(k, nbins, ncheb, 1e-250, want_sorted=True)
            torch.cuda.synchronize()
            assert torch.equal(srt, s_r)
            c, cr = coef.cpu().numpy(), c_r.cpu().numpy()
            assert np.max(np.abs(c - cr) / np.max(np.abs(cr), axis=1, keepdims=True)) <= 1e-9
            m, mr = mean.cpu().numpy(), m_r.cpu().numpy()
            assert np.max(np.abs(m - mr) / mr) <= 1e-12
        # beyond the stated maximum: rejected before any GPU work
        big = torch.ones(2 * 12289, dtype=torch.float64, device="cuda")
        st, _, _, _ = _call_static(helk, big, 2, 20, 1e-250, stream)
        assert st == helk.HELK_ERR_INVALID_ARG
        st, _, _, _ = _call_static(helk, big[:100], 1, 33, 1e-250, stream)
        assert st == helk.HELK_ERR_INVALID_ARG
    finally:
        ctx.close()
