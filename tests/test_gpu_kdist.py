"""GPU parity of the k-distribution stage (Sec. 2.2, 2.6).

Sorted values: bit-exact against the oracle's library sort on identical
input, on every sort path of a bin: the bucket sort (a crowded bucket of one
value, e.g. a run of zeros, ranked by position; one crowded by distinct
values sends the bin to radix passes), for bins in shared memory and for
bins in the global buffers.  Chebyshev coefficients: the GPU applies the pseudo-inverse of the
design matrix shared by all bins (one Householder QR per bin size), the
oracle runs a Householder QR per bin; both are backward stable and the basis
is well conditioned at the workloads' bin sizes (cond(A) ~ 5), so the
coefficient vectors agree to ~1e-13 of their norm; the bar is 1e-9 of max|c|
per bin.
Bin means: 1e-12 relative (summation order only).  When N_b is close to
n_cheb the least-squares problem itself becomes ill-conditioned (uniform
abscissae: cond(A) = 2.9e8 for 32 points and 32 coefficients), and any two
backward-stable solvers then differ by up to ~eps cond(A); the bar becomes
max(1e-9, 100 eps cond(A)).
"""
import numpy as np
import pytest

import oracle
from paper_1503_03806_gb300 import synth
from tests.helpers import NTHREADS, assert_rel

pytestmark = pytest.mark.gpu

RTOL_COEF = 1e-9


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


def check_kdist(ctx, kappa, nbins, ncheb, floor=1e-250, on_host=False):
    import torch
    kt = torch.from_numpy(kappa).cuda()
    coef, mean, srt = ctx.kdist(kt, nbins, ncheb, floor, want_sorted=True, on_host=on_host)
    if not on_host:
        coef, mean = coef.cpu().numpy(), mean.cpu().numpy()
    srt = srt.cpu().numpy()
    s_or, c_or, m_or = oracle.kdist(kappa, nbins, ncheb, floor)
    assert np.array_equal(srt.view(np.uint64), s_or.view(np.uint64)), "sorted values differ"
    scale = np.max(np.abs(c_or), axis=1, keepdims=True)
    err = np.max(np.abs(coef - c_or) / scale)
    nb = kappa.shape[0] // nbins
    g = (np.arange(nb) + 0.5) / nb
    cond = np.linalg.cond(np.polynomial.chebyshev.chebvander(2 * g - 1, ncheb - 1))
    tol = max(RTOL_COEF, 100 * np.finfo(float).eps * cond)
    assert err <= tol, (err, tol, cond)
    assert_rel(mean, m_or, 1e-12, "bin mean")
    return err


@pytest.mark.parametrize("nbins,nb", [(1, 100), (7, 1000), (3, 10000), (2, 12345), (2, 30000),
                                      (5, 20)])
def test_sort_and_fit_random(ctx, nbins, nb):
    k = synth.uniform_kappa(nbins * nb, nb + nbins)
    check_kdist(ctx, k, nbins, min(20, nb))


def test_ties_zeros_and_floor(ctx):
    rng = np.random.default_rng(3)
    k = synth.uniform_kappa(4 * 5000, 4)
    k[:3000] = 0.0                       # empty points (ln of the floor)
    k[6000:9000] = 1e-21                 # one repeated value
    k[10000:15000] = rng.choice([1e-22, 2e-22, 3e-22], 5000)
    check_kdist(ctx, k, 4, 20, floor=1e-40)


def _tied_high_words(n, group, seed):
    """Opacities in groups of `group` values that share the high 32 bits
    (sign, exponent, top 20 fraction bits) and differ in the low 32, in
    random order: the order inside each group is decided by the low word."""
    rng = np.random.default_rng(seed)
    base = synth.uniform_kappa(n // group + 1, seed).view(np.uint64) & np.uint64(0xFFFFFFFF00000000)
    hi = np.repeat(base, group)[:n]
    lo = rng.integers(0, 2**32, n, dtype=np.uint64)
    bits = hi | lo
    rng.shuffle(bits)
    return bits.view(np.float64)


def _with_zeros(k, nbins, nzero):
    """The same opacities with the first nzero points of every bin set to 0:
    more than 512 equal keys fill one bucket of the bucket sort (ranked by
    position in a shared-memory bin; the radix passes for a bin in the
    global buffers)."""
    k = k.copy().reshape(nbins, -1)
    k[:, :nzero] = 0.0
    return k.reshape(-1)


def _with_crowd(k, nbins, ncrowd, seed):
    """The same opacities with ncrowd points of every bin replaced by
    distinct values within 1e-9 of each other (and of 1e-20), in random
    places: more than 512 different keys in one bucket, so the bin takes
    the radix passes."""
    rng = np.random.default_rng(seed)
    k = k.copy().reshape(nbins, -1)
    for b in range(nbins):
        at = rng.choice(k.shape[1], ncrowd, replace=False)
        k[b, at] = 1e-20 * (1.0 + 1e-9 * rng.random(ncrowd))
    return k.reshape(-1)


def test_high_word_ties_short_runs(ctx):
    # runs of 2..5 keys equal in the high word: in one bucket of the bucket
    # sort; beside a run of zeros; on the radix passes (a crowded bucket)
    for group in (2, 3, 5):
        k = _tied_high_words(4 * 9000, group, 20 + group)
        check_kdist(ctx, k, 4, 20)
        check_kdist(ctx, _with_zeros(k, 4, 600), 4, 20, floor=1e-40)
        check_kdist(ctx, _with_crowd(k, 4, 700, group), 4, 20)


def test_high_word_ties_long_runs(ctx):
    # runs of 200 in one bucket of the bucket sort; the same beside a long
    # run of zeros, and on the radix passes
    k = _tied_high_words(3 * 8000, 200, 31)
    check_kdist(ctx, k, 3, 20)
    check_kdist(ctx, _with_zeros(k, 3, 600), 3, 20, floor=1e-40)
    check_kdist(ctx, _with_crowd(k, 3, 600, 31), 3, 20)
    k = _tied_high_words(2 * 6000, 2, 32)
    k[:2000] = 0.0
    check_kdist(ctx, k, 2, 20, floor=1e-40)


def test_crowded_bucket_takes_the_radix_passes(ctx):
    # more than 512 distinct keys in one bucket (with and without a run of
    # zeros in another), bins of the workloads' size and a ragged one
    for nbins, nb in [(3, 10000), (2, 12345), (5, 1031)]:
        k = _with_crowd(synth.uniform_kappa(nbins * nb, nb), nbins, 520 if nb < 2000 else 1500, nb)
        check_kdist(ctx, k, nbins, 20)
        check_kdist(ctx, _with_zeros(k, nbins, 513), nbins, 20, floor=1e-40)
    # every bucket crowded but one value each: ranked by position
    k = np.repeat(synth.uniform_kappa(8, 5), 1000)
    np.random.default_rng(6).shuffle(k)
    check_kdist(ctx, k, 2, 20)


def test_constant_bin_skips_all_passes(ctx):
    k = np.full(3 * 777, 3.5e-21)
    check_kdist(ctx, k, 3, 8)


def test_ncheb_extremes(ctx):
    k = synth.uniform_kappa(2 * 64, 9)
    check_kdist(ctx, k, 2, 1)
    check_kdist(ctx, k, 2, 32)
    check_kdist(ctx, synth.uniform_kappa(3 * 32, 10), 3, 32)


def test_host_outputs(ctx):
    check_kdist(ctx, synth.uniform_kappa(10 * 3000, 11), 10, 20, on_host=True)


def test_opacity_then_kdist_on_small_workload(ctx):
    # the whole path at the 1e4-line workload: oracle kappa -> oracle tables,
    # GPU kappa -> GPU tables (inputs differ at ~1e-15, tables at ~1e-13)
    w = synth.WORKLOADS["small"]
    lines = synth.workload_lines("small")
    ctx.upload(lines)
    k = ctx.opacity(w["T"][0], w["P_atm"][0], w["mass"], w["cut"],
                    (w["nu_min"], w["dnu"], w["ngrid"]))
    coef, mean, _ = ctx.kdist(k, w["nbins"], w["ncheb"])
    ko, _, _ = oracle.opacity(lines, oracle.Condition(w["T"][0], w["P_atm"][0], w["mass"],
                                                      w["nu_min"], w["dnu"], w["ngrid"],
                                                      oracle.CUT_ABS, w["cut"][1]),
                              nthreads=NTHREADS)
    _, c_or, m_or = oracle.kdist(ko, w["nbins"], w["ncheb"])
    c = coef.cpu().numpy()
    scale = np.max(np.abs(c_or), axis=1, keepdims=True)
    assert np.max(np.abs(c - c_or) / scale) <= RTOL_COEF
    assert_rel(mean.cpu().numpy(), m_or, 1e-9, "bin mean")


def test_invalid_arguments(ctx):
    import torch
    from paper_1503_03806_gb300 import helk
    k = torch.ones(100, dtype=torch.float64, device="cuda")
    for nbins, ncheb, floor in [(3, 5, 1e-250), (10, 11, 1e-250), (1, 33, 1e-250), (1, 0, 1e-250),
                                (1, 5, 0.0)]:
        with pytest.raises(helk.HelkError) as e:
            ctx.kdist(k, nbins, ncheb, floor)
        assert e.value.status == helk.HELK_ERR_INVALID_ARG


def test_global_path_bucket_and_radix(ctx):
    # bins of 30000 points (sorted through the global buffers): the bucket
    # sort, and, with more than 512 equal keys in a bucket, the radix passes
    k = synth.uniform_kappa(2 * 30000, 31)
    check_kdist(ctx, k, 2, 20)
    check_kdist(ctx, _with_zeros(k, 2, 1000), 2, 20, floor=1e-40)
    check_kdist(ctx, _tied_high_words(3 * 30000, 3, 32), 3, 20)
