"""The GPU detector noise judged statistically against the FP64 oracle's law.

The kernel and the oracle draw their counts by different algorithms and in
different precisions (the kernel: float32 decisions, a 24-bit uniform, a
rejection sampler from lambda = 10 on; the oracle: FP64 inversion of the Poisson
CDF), so their draws are compared as distributions, over 1000 frames:

  * every pixel's sample mean and variance against lambda (+ sigma^2) with a
    z-bound (4096 pixels: the bound of 6 standard errors leaves a false-alarm
    probability of about 1e-5 for the whole test);
  * the pooled counts of each lambda level (512 pixels x 1000 frames) against
    the oracle's FP64 Poisson pmf by a chi-square goodness-of-fit test
    (bins merged to expected counts >= 20, p > 1e-6);
  * read noise on unlit pixels against N(0, sigma^2) by Kolmogorov-Smirnov.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LEVELS = [0.0, 0.1, 1.0, 9.99, 10.0, 10.01, 100.0, 1000.0]   # lambda of each 512-pixel block
N_FRAMES = 1000
SEED = 2024


def _draw(read_noise_e):
    import torch
    from paper_1607_07624_gb300 import pas
    lam = np.repeat(np.array(LEVELS, dtype=np.float32), 512)
    ctx = pas.pas_ctx_create()
    try:
        d_in = torch.as_tensor(lam).cuda()
        out = torch.zeros(N_FRAMES, lam.size, device="cuda")
        for t in range(N_FRAMES):
            # one photon per "pupil pixel": lambda_p equals the input value
            pas.pas_ccd_noise(ctx, d_in, out[t], 1.0, 1, read_noise_e, SEED, t)
        torch.cuda.synchronize()
        return lam.astype(np.float64), out.cpu().numpy().astype(np.float64)
    finally:
        pas.pas_ctx_destroy(ctx)


def _chi2_against_pmf(x, lam):
    from scipy.stats import chi2
    from oracle import noise as nz
    n = x.size
    kmax = int(max(x.max(), lam + 12 * math.sqrt(lam) + 12))
    k = np.arange(kmax + 1)
    expected = n * nz.poisson_pmf(k, lam)
    observed = np.bincount(x.astype(np.int64), minlength=kmax + 1)[:kmax + 1].astype(np.float64)
    # merge neighbouring bins from both tails towards the mode until each holds >= 20
    bins_o, bins_e, acc_o, acc_e = [], [], 0.0, 0.0
    for o, e in zip(observed, expected):
        acc_o += o
        acc_e += e
        if acc_e >= 20.0:
            bins_o.append(acc_o)
            bins_e.append(acc_e)
            acc_o = acc_e = 0.0
    bins_o[-1] += acc_o + (n - observed.sum())
    bins_e[-1] += acc_e + (n - expected.sum())
    bins_o, bins_e = np.array(bins_o), np.array(bins_e)
    stat = float(np.sum((bins_o - bins_e) ** 2 / bins_e))
    return stat, float(chi2.sf(stat, bins_o.size - 1)), bins_o.size


def test_photon_noise_law_matches_fp64_poisson():
    lam, x = _draw(0.0)
    assert np.all(x == np.round(x)) and np.all(x >= 0)
    assert np.all(x[:, lam == 0.0] == 0.0)
    F = N_FRAMES
    lit = lam > 0
    m = x[:, lit].mean(axis=0)
    v = x[:, lit].var(axis=0, ddof=1)
    L = lam[lit]
    z_mean = (m - L) / np.sqrt(L / F)
    z_var = (v - L) / np.sqrt((L + 2.0 * L * L) / F)
    assert np.max(np.abs(z_mean)) < 6.0, np.max(np.abs(z_mean))
    assert np.max(np.abs(z_var)) < 6.0, np.max(np.abs(z_var))
    for level in LEVELS[1:]:
        lv = float(np.float32(level))            # the float32 value the kernel received
        sel = lam == lv
        assert sel.sum() == 512
        stat, p, nb = _chi2_against_pmf(x[:, sel].ravel(), lv)
        assert p > 1e-6, (level, stat, nb, p)


def test_read_noise_and_photon_noise_together():
    from scipy.stats import kstest, norm
    sigma = 0.5
    lam, x = _draw(sigma)
    F = N_FRAMES
    m = x.mean(axis=0)
    v = x.var(axis=0, ddof=1)
    var = lam + sigma ** 2
    mu4 = lam + 3.0 * lam ** 2 + 6.0 * lam * sigma ** 2 + 3.0 * sigma ** 4   # central 4th moment
    z_mean = (m - lam) / np.sqrt(var / F)
    z_var = (v - var) / np.sqrt((mu4 - var ** 2) / F)
    assert np.max(np.abs(z_mean)) < 6.0, np.max(np.abs(z_mean))
    assert np.max(np.abs(z_var)) < 6.0, np.max(np.abs(z_var))
    # unlit pixels: read noise alone
    r = x[:, lam == 0.0].ravel()
    assert kstest(r, norm(loc=0.0, scale=sigma).cdf).pvalue > 1e-6
    # lit pixels: count + Gaussian, so x - sigma g is not an integer in general
    assert np.mean(x[:, lam > 0] != np.round(x[:, lam > 0])) > 0.99


def test_noise_is_reproducible_by_counter():
    import torch
    from paper_1607_07624_gb300 import pas
    ctx = pas.pas_ctx_create()
    try:
        d_in = torch.full((4096,), 37.5, device="cuda")
        a, b, c = (torch.zeros_like(d_in) for _ in range(3))
        pas.pas_ccd_noise(ctx, d_in, a, 1.0, 1, 0.5, SEED, 41)
        pas.pas_ccd_noise(ctx, d_in, b, 1.0, 1, 0.5, SEED, 41)
        pas.pas_ccd_noise(ctx, d_in, c, 1.0, 1, 0.5, SEED, 42)
        torch.cuda.synchronize()
        assert torch.equal(a, b) and not torch.equal(a, c)
        # photons <= 0: no detector model, the frame is left as it is
        pas.pas_ccd_noise(ctx, d_in, c, 0.0, 1, 0.5, SEED, 42)
        torch.cuda.synchronize()
        assert torch.equal(c, d_in)
    finally:
        pas.pas_ctx_destroy(ctx)
