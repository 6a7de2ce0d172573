"""Oracle Shack-Hartmann wavefront sensor: lenslet spots, detector frame, centroid slopes.

Test infrastructure only (imported by tests/, the smoke check and bench.py's CPU
baseline), never by the product path.

Paper passages: the Shack-Hartmann sensor is named beside the pyramid as a sensor of
the framework and as one of its GPU areas ("Pyramid and Shack Hartmann propagation
(from wavefront to detector plane)", Sec. GPU acceleration); the paper gives no
parameter or formula for it. Readings (textbook Shack-Hartmann model):

  * an n_sub x n_sub lenslet array on the Np x Np pupil, lenslet (r, c) covering the
    b x b pupil pixels [r b, (r+1) b) x [c b, (c+1) b), b = Np / n_sub an integer;
  * the lenslet's field E = A exp(2 pi i opd / lambda) (A = the pupil stop of the
    optics oracle) zero-padded to M x M, M = ovs b (ovs = 2: Nyquist-sampled spots);
  * spot I(k, l) = |F(k - M/2, l - M/2)|^2 / M^2 with F the plain 2-D DFT, so the
    zero frequency sits at pixel (M/2, M/2) and a spot's total equals the number of
    pupil pixels of its lenslet (Parseval); one pixel is lambda / (ovs d), d the
    lenslet size;
  * the detector frame tiles the spots: lenslet (r, c) occupies rows [r M, (r+1) M)
    and columns [c M, (c+1) M);
  * slopes = centre of gravity (sum I (k - M/2), sum I (l - M/2)) / sum I in pixels,
    x along axis 0 and y along axis 1, for the valid lenslets (the pyramid's
    geometric rule) in row-major order, layout [x; y], minus the reference slopes
    of a flat wavefront.
"""
from __future__ import annotations

import numpy as np

from oracle.optics import pupil_mask, valid_subapertures


def lenslet_spot(E_sub: np.ndarray, M: int) -> np.ndarray:
    """|fftshift(DFT2(E padded to M x M))|^2 / M^2 for one lenslet field (b x b)."""
    b = E_sub.shape[0]
    pad = np.zeros((M, M), dtype=np.complex128)
    pad[:b, :b] = E_sub
    F = np.fft.fftshift(np.fft.fft2(pad))
    return np.abs(F) ** 2 / float(M * M)


def sh_frame(opd_nm: np.ndarray, wavelength_nm: float, obs: float, n_sub: int, ovs: int) -> np.ndarray:
    """Detector frame (n_sub M)^2 of tiled spots."""
    opd = np.asarray(opd_nm, dtype=np.float64)
    Np = opd.shape[0]
    assert Np % n_sub == 0
    b = Np // n_sub
    M = ovs * b
    E = pupil_mask(Np, obs) * np.exp(2j * np.pi * opd / wavelength_nm)
    frame = np.zeros((n_sub * M, n_sub * M))
    for r in range(n_sub):
        for c in range(n_sub):
            frame[r * M:(r + 1) * M, c * M:(c + 1) * M] = lenslet_spot(E[r * b:(r + 1) * b, c * b:(c + 1) * b], M)
    return frame


def centroids(frame: np.ndarray, n_sub: int) -> tuple[np.ndarray, np.ndarray]:
    """Centre of gravity of every lenslet's spot about (M/2, M/2), in pixels
    (n_sub x n_sub arrays; NaN where a spot has no light)."""
    M = frame.shape[0] // n_sub
    k = np.arange(M) - M / 2.0
    cx = np.full((n_sub, n_sub), np.nan)
    cy = np.full((n_sub, n_sub), np.nan)
    for r in range(n_sub):
        for c in range(n_sub):
            I = frame[r * M:(r + 1) * M, c * M:(c + 1) * M]
            s = I.sum()
            if s > 0:
                cx[r, c] = (I.sum(axis=1) * k).sum() / s
                cy[r, c] = (I.sum(axis=0) * k).sum() / s
    return cx, cy


def sh_slopes(frame: np.ndarray, valid: np.ndarray, n_sub: int, ref=None) -> np.ndarray:
    """[x; y] centroids of the valid lenslets (row-major indices r n_sub + c) minus ref."""
    cx, cy = centroids(frame, n_sub)
    s = np.concatenate([cx.ravel()[valid], cy.ravel()[valid]])
    return s if ref is None else s - ref


def sh_measure(opd_nm, wavelength_nm: float, obs: float, n_sub: int, ovs: int, valid=None, ref=None):
    """opd -> (frame, slopes); valid defaults to the geometric rule."""
    Np = np.shape(opd_nm)[0]
    if valid is None:
        valid = valid_subapertures(Np, obs, n_sub)
    frame = sh_frame(opd_nm, wavelength_nm, obs, n_sub, ovs)
    return frame, sh_slopes(frame, valid, n_sub, ref)
