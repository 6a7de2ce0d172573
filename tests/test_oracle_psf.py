"""Pins of the oracle PSF camera (oracle/psf.py) against what the mathematics fixes:
a brute-force DFT, Parseval, the diffraction-limited peak and the Airy profile, the
exact shift of a tilt, the reflection of the conjugate field, and Marechal's law."""
import math

import numpy as np
import pytest

from oracle import optics as op
from oracle import psf as ps

LAM = 1650.0


def _random_opd(Np, rms_nm, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((Np, Np)) * rms_nm


@pytest.mark.parametrize("Np,nd,obs", [(4, 2, 0.0), (6, 3, 0.1), (8, 2, 0.25)])
def test_psf_equals_brute_force_dft(Np, nd, obs):
    """F(p, q) = sum_ij E(i, j) exp(-2 pi i (p i + q j) / N) by four nested sums,
    zero frequency moved to (N/2, N/2) by index arithmetic."""
    opd = _random_opd(Np, 400.0, Np + nd)
    A = op.pupil_mask(Np, obs)
    N = nd * Np
    n_pup = A.sum()
    out = np.zeros((N, N))
    for k in range(N):
        for l in range(N):
            p, q = (k - N // 2) % N, (l - N // 2) % N
            s = 0j
            for i in range(Np):
                for j in range(Np):
                    if A[i, j]:
                        s += np.exp(2j * math.pi * opd[i, j] / LAM) * np.exp(-2j * math.pi * (p * i + q * j) / N)
            out[k, l] = abs(s) ** 2 / n_pup ** 2
    assert np.max(np.abs(ps.psf(opd, LAM, obs, nd) - out)) < 1e-12


@pytest.mark.parametrize("Np,nd,obs", [(32, 4, 0.1), (24, 8, 0.0)])
def test_flat_wavefront_peak_parseval_and_symmetry(Np, nd, obs):
    N = nd * Np
    flat = np.zeros((Np, Np))
    P = ps.psf(flat, LAM, obs, nd)
    n_pup = op.pupil_mask(Np, obs).sum()
    assert ps.strehl(flat, LAM, obs) == 1.0
    assert abs(P[N // 2, N // 2] - 1.0) < 1e-12 and np.argmax(P) == (N // 2) * N + N // 2
    # Parseval for the plain DFT: sum |F|^2 = N^2 sum |E|^2
    assert abs(P.sum() - N * N / n_pup) < 1e-9 * N * N / n_pup
    # real field: point symmetry about the zero frequency
    idx = (N - np.arange(N)) % N      # k -> N - k is the reflection about N/2
    assert np.max(np.abs(P - P[idx][:, idx])) < 1e-12


def test_conjugate_field_gives_the_point_reflected_psf():
    Np, nd, N = 16, 4, 64
    opd = _random_opd(Np, 300.0, 3)
    idx = (N - np.arange(N)) % N
    assert np.max(np.abs(ps.psf(-opd, LAM, 0.1, nd) - ps.psf(opd, LAM, 0.1, nd)[idx][:, idx])) < 1e-12


@pytest.mark.parametrize("m,axis", [(1, 0), (-2, 0), (3, 1)])
def test_tilt_of_m_cycles_shifts_the_psf_by_m_nd_pixels(m, axis):
    """A phase ramp of m whole waves across the Np pixels moves the PSF by exactly
    m nd pixels towards positive frequency along that axis."""
    Np, nd, obs = 20, 6, 0.1
    i = np.arange(Np, dtype=np.float64)
    ramp = m * LAM * i / Np
    opd = np.repeat(ramp[:, None], Np, 1) if axis == 0 else np.repeat(ramp[None, :], Np, 0)
    P0 = ps.psf(np.zeros((Np, Np)), LAM, obs, nd)
    P1 = ps.psf(opd, LAM, obs, nd)
    assert np.max(np.abs(P1 - np.roll(P0, m * nd, axis=axis))) < 1e-12


def test_disc_gives_the_airy_profile():
    """Unobstructed disc of 96 px, nd = 8: the profile through the centre against
    [2 J1(pi rho) / (pi rho)]^2, rho = offset / nd in lambda/D (first zero 1.22)."""
    from scipy.special import j1
    Np, nd = 96, 8
    N = nd * Np
    P = ps.psf(np.zeros((Np, Np)), LAM, 0.0, nd)
    prof = P[N // 2, N // 2:N // 2 + 3 * nd]
    rho = np.arange(prof.size) / nd
    x = np.pi * np.where(rho == 0, 1e-30, rho)
    airy = np.where(rho == 0, 1.0, (2 * j1(x) / x) ** 2)
    assert np.max(np.abs(prof - airy)) < 2e-3          # measured 5.1e-4; nd halved gives 0.50
    # the first dark ring between 1.1 and 1.35 lambda/D
    k0 = np.argmin(prof[: 2 * nd])
    assert 1.1 <= k0 / nd <= 1.35 and prof[k0] < 5e-3


def test_marechal_small_aberration():
    """SR = |<exp(i phi)>|^2 = exp(-sigma^2) + O(sigma^4) for a small piston-free phase."""
    Np = 48
    A = op.pupil_mask(Np, 0.1)
    rng = np.random.default_rng(11)
    phi = rng.standard_normal((Np, Np))
    phi -= phi[A].mean()
    phi *= 0.05 / np.sqrt(np.mean(phi[A] ** 2))
    opd = phi * LAM / (2 * np.pi)
    sr = ps.strehl(opd, LAM, 0.1)
    assert abs(sr - math.exp(-0.05 ** 2)) < 1e-5
    P = ps.psf(opd, LAM, 0.1, 2)
    assert abs(P[Np, Np] - sr) < 1e-12


def test_integrated_psf_sums_from_the_start_step():
    Np, nd = 12, 2
    opds = [_random_opd(Np, 100.0 * (t + 1), 20 + t) for t in range(4)]
    tot = ps.integrated_psf(opds, LAM, 0.1, nd, start=1)
    ref = sum(ps.psf(o, LAM, 0.1, nd) for o in opds[1:])
    assert np.max(np.abs(tot - ref)) < 1e-12
