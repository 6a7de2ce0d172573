"""Oracle PSF camera: point-spread function and Strehl ratio of the residual field.

Test infrastructure only (imported by tests/, the smoke check and bench.py's CPU
baseline), never by the product path.

Paper passages: the camera object (Table 1 ``camera``: wavelengthInNm, nd "padding
coefficient for PSF computation", start_time "PSF integration start time"), the PSF
object fed with the residual electric field and giving the Strehl ratio and the
integrated PSF (Table 2: psf.in_ef, psf.out_sr, psf.out_int_psf), and the GPU area
"PSF generation from residual wavefront" (Sec. GPU acceleration). The paper gives no
formula. Readings (textbook Fourier optics):

  * field E = A exp(2 pi i opd / lambda) on the Np x Np pupil (A = the pupil stop of
    the optics oracle), zero-padded to an N x N grid with N = nd * Np;
  * PSF(p, q) = |F(p, q)|^2 / (sum A)^2 with F the plain 2-D DFT
    F(p, q) = sum_{i,j} E(i, j) exp(-2 pi i (p i + q j) / N), indices shifted so
    that the zero frequency sits at (N/2, N/2) (numpy's fftshift); a diffraction-
    limited pupil then peaks at exactly 1 and one pixel is lambda / (nd D);
  * Strehl ratio SR = |sum A exp(i phi)|^2 / (sum A)^2, the PSF value at the zero
    frequency;
  * the integrated PSF is the sum of the per-step PSFs from the start step on.
"""
from __future__ import annotations

import numpy as np

from oracle.optics import pupil_mask


def field(opd_nm: np.ndarray, wavelength_nm: float, obs: float) -> np.ndarray:
    """E = A exp(2 pi i opd / lambda) on the pupil (complex128, Np x Np)."""
    opd = np.asarray(opd_nm, dtype=np.float64)
    A = pupil_mask(opd.shape[0], obs).astype(np.float64)
    return A * np.exp(2j * np.pi * opd / wavelength_nm)


def psf(opd_nm: np.ndarray, wavelength_nm: float, obs: float, nd: int) -> np.ndarray:
    """Normalised PSF on the nd Np x nd Np grid, zero frequency at (N/2, N/2)."""
    E = field(opd_nm, wavelength_nm, obs)
    Np = E.shape[0]
    N = nd * Np
    pad = np.zeros((N, N), dtype=np.complex128)
    pad[:Np, :Np] = E
    F = np.fft.fftshift(np.fft.fft2(pad))
    n_pup = np.sum(np.abs(E) > 0)
    return np.abs(F) ** 2 / float(n_pup) ** 2


def strehl(opd_nm: np.ndarray, wavelength_nm: float, obs: float) -> float:
    """|sum A exp(i phi)|^2 / (sum A)^2."""
    E = field(opd_nm, wavelength_nm, obs)
    n_pup = np.sum(np.abs(E) > 0)
    return float(np.abs(E.sum()) ** 2 / float(n_pup) ** 2)


def integrated_psf(opds_nm, wavelength_nm: float, obs: float, nd: int, start: int = 0) -> np.ndarray:
    """Sum of the PSFs of the steps t >= start of a sequence of residual OPDs."""
    out = None
    for t, opd in enumerate(opds_nm):
        if t < start:
            continue
        p = psf(opd, wavelength_nm, obs, nd)
        out = p if out is None else out + p
    return out
