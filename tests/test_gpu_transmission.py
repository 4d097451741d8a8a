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


def _direct(ctx, k_bins, m):
    import torch
    k = np.ascontiguousarray(np.asarray(k_bins, dtype=np.float64))
    nbins = k.shape[0]
    srt = torch.from_numpy(k.reshape(-1)).cuda()
    direct, _ = ctx.transmission(nbins, np.asarray(m, dtype=np.float64), sorted_k=srt)
    return direct.cpu().numpy()


def test_direct_terms_against_exp(ctx):
    # bins (0, 1) and (1, 2): T = (1 + e^-m)/2 and e^-m (1 + e^-m)/2 over the
    # whole range of the float-float exponential (d in [0, 87)) and beyond
    m = np.concatenate([[0.0, 1e-300, 1e-20, 1e-9], np.linspace(0.0, 90.0, 3001)[1:],
                        np.logspace(-6, 2.5, 500)])
    got = _direct(ctx, [[0.0, 1.0], [1.0, 2.0]], m)
    want0 = (1.0 + np.exp(-m)) / 2.0
    want1 = np.exp(-m) * (1.0 + np.exp(-m)) / 2.0
    np.testing.assert_allclose(got[0], want0, rtol=2e-14, atol=0)
    np.testing.assert_allclose(got[1], want1, rtol=1e-13, atol=1e-300)


def test_direct_edge_bins_against_oracle(ctx):
    # zeros and ties, differences spanning more than 2^100 (the FP64 terms),
    # huge and subnormal values, a constant bin, an unsorted bin and one with
    # a negative value (both summed plainly in FP64), m from 0 to 1e300
    rng = np.random.default_rng(77)
    nb = 4096
    bins = []
    b = np.sort(10.0 ** rng.uniform(-30, -18, nb)); b[:700] = 0.0; b[700:900] = b[700]
    bins.append(b)
    b = np.sort(np.concatenate([10.0 ** rng.uniform(-60, -50, 100), 10.0 ** rng.uniform(-18, -17, nb - 100)]))
    bins.append(b)
    bins.append(np.sort(10.0 ** rng.uniform(280, 300, nb)))
    b = np.sort(10.0 ** rng.uniform(-320, -300, nb)); bins.append(b)
    bins.append(np.full(nb, 3.5e-21))
    bins.append(10.0 ** rng.uniform(-25, -20, nb))                      # unsorted
    b = np.sort(10.0 ** rng.uniform(-25, -20, nb)); b[5] = -1e-30; bins.append(b)  # negative
    k = np.stack(bins)
    m = np.concatenate([[0.0], np.logspace(-310, 300, 400)])
    got = _direct(ctx, k, m)
    d_or, _ = oracle.transmission(k.reshape(-1), k.shape[0], m)
    np.testing.assert_allclose(got, d_or, rtol=1e-12, atol=1e-300)


def test_fit_paths_against_oracle(ctx):
    # the fit's float-float sum (ng points in shared memory) and its plain
    # FP64 sum for the largest ng; coefficients set directly.  Both sides
    # evaluate k(g) = exp(sum c_k T_k) in FP64 but round differently (the GPU
    # contracts multiply-adds): ~1.5e-14 relative in k, which the exponent
    # multiplies by k m ~ |ln T|, so the bar is 1e-12 + 2e-14 |ln T|
    import torch
    rng = np.random.default_rng(78)
    nbins, ncheb = 3, 12
    c = rng.normal(0.0, 1.0, (nbins, ncheb))
    c[:, 0] = [-50.0, -45.0, -40.0]
    c[:, 1] = [3.0, 6.0, 10.0]
    m = np.concatenate([[0.0], np.logspace(10, 30, 300)])
    ct = torch.from_numpy(c).cuda()
    k_dummy = np.zeros(nbins * 16)
    for ng in (1000, 16384):
        _, fit = ctx.transmission(nbins, m, coeffs=ct, ng=ng)
        _, f_or = oracle.transmission(k_dummy, nbins, m, coeffs=c, ng=ng)
        f = fit.cpu().numpy()
        pos = f_or > 1e-300
        assert np.all(np.abs(f[~pos]) <= 1e-299)
        rel = np.abs(f[pos] / f_or[pos] - 1.0)
        assert np.all(rel <= 1e-12 + 2e-14 * np.abs(np.log(f_or[pos]))), rel.max()
