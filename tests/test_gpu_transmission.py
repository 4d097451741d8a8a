"""Transmission of the k-distribution bins (Sec. 2.1, Eq. for T) on the GPU
against the oracle: from the sorted values (midpoint rule on g) and from
the Chebyshev fit (midpoint rule on ng points).  Direct: 1e-12 relative
(exp implementations and summation order only).  Fit: each side uses its own
coefficients (GPU vs oracle, equal to ~1e-13 of their size), which moves
ln T(m) by up to |d ln k| k m <= |d ln k| |ln T|: the bar is
|d ln T| <= 1e-10 (1 + |ln T|)."""
import numpy as np
import pytest

import oracle
from paper_1503_03806_gb300 import synth
from tests.helpers import NTHREADS

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


def test_transmission_matches_oracle(ctx):
    import torch
    lines = synth.random_lines(600, 501, 0.0, 100.0)
    cond = oracle.Condition(1500.0, 1.0, 18.0, 0.0, 0.01, 10000, oracle.CUT_ABS, 10.0)
    k, _, _ = oracle.opacity(lines, cond, nthreads=NTHREADS)
    nbins, ncheb = 10, 20
    m = np.logspace(16, 26, 1000)
    kt = torch.from_numpy(k).cuda()
    coef, _, srt = ctx.kdist(kt, nbins, ncheb, want_sorted=True)
    direct, fit = ctx.transmission(nbins, m, sorted_k=srt, coeffs=coef, ng=64)
    s_or = oracle.sort_bins(k, nbins)
    c_or, _ = oracle.chebfit(s_or, nbins, ncheb)
    d_or, f_or = oracle.transmission(s_or, nbins, m, coeffs=c_or, ng=64)
    np.testing.assert_allclose(direct.cpu().numpy(), d_or, rtol=1e-12, atol=1e-300)
    fg = fit.cpu().numpy()
    pos = f_or > 0
    assert np.array_equal(pos, fg > 0)
    dlog = np.abs(np.log(fg[pos]) - np.log(f_or[pos]))
    assert np.all(dlog <= 1e-10 * (1 + np.abs(np.log(f_or[pos])))), dlog.max()
    # Sec. 2.1: the sorted-sample transmission is the band mean of the unsorted bin
    band = np.exp(-np.outer(k, m)).reshape(nbins, -1, m.size).mean(axis=1)
    np.testing.assert_allclose(direct.cpu().numpy(), band, rtol=1e-12, atol=1e-300)
    # and the 20-coefficient resampling changes it by << 1 % (Sec. 3.2)
    assert np.max(np.abs(fit.cpu().numpy() - direct.cpu().numpy())) < 1e-2


def test_transmission_arguments(ctx):
    import torch
    from paper_1503_03806_gb300 import helk
    srt = torch.ones(100, dtype=torch.float64, device="cuda")
    with pytest.raises(helk.HelkError):
        ctx.transmission(2, [-1.0], sorted_k=srt)
    with pytest.raises(helk.HelkError):
        ctx.transmission(2, [float("nan")], sorted_k=srt)
