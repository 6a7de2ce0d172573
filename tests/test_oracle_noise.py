"""Pins of the oracle's FP64 detector noise against the Poisson and normal laws.

The sampler inverts the Poisson CDF (scipy's regularised incomplete gamma); these
tests tie it to things it does not use: the pmf summed term by term with the
recurrence p_k = p_(k-1) lambda / k, the moments of the law, a chi-square fit of
its draws, and the normal law of the Box-Muller read noise.
"""
import math

import numpy as np
import pytest

from oracle import noise as nz


def _cdf_by_recurrence(k, lam):
    p = math.exp(-lam)
    terms = [p]
    for j in range(1, k + 1):
        p *= lam / j
        terms.append(p)
    return math.fsum(terms)


@pytest.mark.parametrize("lam", [0.3, 4.0, 25.0, 90.0])
def test_inverse_cdf_lands_on_the_cdf_step(lam):
    u = np.random.default_rng(5).random(400) * (1 - 2e-9) + 1e-9
    k = nz.poisson_inverse_cdf(u, lam)
    for ui, ki in zip(u, k):
        hi = _cdf_by_recurrence(int(ki), lam)
        lo = _cdf_by_recurrence(int(ki) - 1, lam) if ki > 0 else 0.0
        assert lo < ui <= hi + 1e-14, (ui, ki, lo, hi)


def test_inverse_cdf_special_values():
    # P(X = 0) = e^-lam: u at or below it gives 0, just above gives 1
    lam = 2.0
    p0 = math.exp(-lam)
    assert nz.poisson_inverse_cdf(np.array([p0 * 0.999999]), lam)[0] == 0
    assert nz.poisson_inverse_cdf(np.array([p0 * 1.000001]), lam)[0] == 1
    # the median of Poisson(lam) lies within [lam - ln 2, lam + 1/3] (Choi 1994)
    for lam in (0.5, 3.7, 40.0, 1000.0):
        med = nz.poisson_inverse_cdf(np.array([0.5]), lam)[0]
        assert lam - math.log(2) - 1e-12 <= med <= lam + 1 / 3 + 1e-12


@pytest.mark.parametrize("lam", [0.1, 2.5, 40.0, 1000.0])
def test_sampler_fits_the_pmf(lam):
    from scipy.stats import chi2
    n = 6000
    x = np.array([nz.poisson(lam, 77, p, 5) for p in range(n)])
    kmax = int(x.max() + 1)
    k = np.arange(kmax + 1)
    e = n * nz.poisson_pmf(k, lam)
    o = np.bincount(x, minlength=kmax + 1)[:kmax + 1].astype(float)
    bo, be, ao, ae = [], [], 0.0, 0.0
    for oi, ei in zip(o, e):
        ao += oi
        ae += ei
        if ae >= 10:
            bo.append(ao)
            be.append(ae)
            ao = ae = 0.0
    bo[-1] += ao
    be[-1] += ae + (n - e.sum())
    bo, be = np.array(bo), np.array(be)
    stat = np.sum((bo - be) ** 2 / be)
    assert chi2.sf(stat, max(1, bo.size - 1)) > 1e-5
    assert abs(x.mean() - lam) < 5 * math.sqrt(lam / n)


def test_pmf_sums_to_one_and_matches_recurrence():
    for lam in (0.2, 7.0, 60.0):
        k = np.arange(0, int(lam + 20 * math.sqrt(lam) + 30))
        p = nz.poisson_pmf(k, lam)
        assert abs(p.sum() - 1.0) < 1e-12
        assert abs(p[5] - (_cdf_by_recurrence(5, lam) - _cdf_by_recurrence(4, lam))) < 1e-13


def test_read_noise_alone_is_normal_and_photons_off_keeps_the_frame():
    from scipy.stats import kstest, norm
    fr = np.zeros((60, 60))
    sigma = 2.0
    x = np.concatenate([nz.apply_noise(fr, 1.0e4, 100, sigma, 9, t).ravel() for t in range(3)])
    assert kstest(x, norm(loc=0.0, scale=sigma).cdf).pvalue > 1e-4
    lit = np.full((4, 4), 3.0)
    assert np.array_equal(nz.apply_noise(lit, 0.0, 16, sigma, 9, 0), lit)
    # lambda = 3 per pixel with read noise: the mean over many pixels
    y = nz.apply_noise(np.full((80, 80), 3.0), 16.0, 16, 0.5, 9, 2)
    assert abs(y.mean() - 3.0) < 5 * math.sqrt(3.25 / y.size)


def test_uniform_is_open_and_full_precision():
    assert 0.0 < nz.uniform(0) < 2.0 ** -32
    assert 1.0 - 2.0 ** -32 < nz.uniform(0xFFFFFFFF) < 1.0
    # 32 bits of the word survive (a 24-bit uniform would merge these two)
    assert nz.uniform(256) != nz.uniform(257)
