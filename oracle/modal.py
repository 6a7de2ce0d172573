"""Oracle modal DM, interaction matrix and reconstructor.

Paper passages: the modal DM (Table 1 ``DM``: type 'zernike', nmodes, npixels,
obsratio), the modal reconstructor with its reconstruction matrix (Table 1
``modalrec.recmat_tag``), the calibration of the reconstruction matrix that the
paper mentions but does not list (Sec. Example), and the GPU area "influence
function multiplication" (Sec. GPU acceleration). Readings:

  * Zernike polynomials in Noll order j = 2 .. n_modes+1 (piston excluded), Noll's
    normalisation, evaluated at pixel centres with rho = 1 at the pupil edge, theta
    from axis 0; then orthonormalised on the annular mask pixels by QR in the same
    column order, scaled so that a unit coefficient is 1 nm RMS over the pupil;
  * push-pull interaction matrix IM[:, m] = (s(+a e_m) - s(-a e_m)) / (2a), with the
    slope reference subtracted, a = 10 nm RMS;
  * reconstruction matrix R = pinv(IM) by FP64 SVD, dropping singular values below
    rcond * s_max.
"""
from __future__ import annotations

import math

import numpy as np

from .atmosphere import von_karman_psd
from .optics import pupil_mask


def noll_to_nm(j: int) -> tuple[int, int]:
    """Noll index j >= 1 -> (n, m); m > 0 cosine (even j), m < 0 sine (odd j)."""
    if j < 1:
        raise ValueError("Noll index starts at 1")
    n = 0
    while (n + 1) * (n + 2) // 2 < j:
        n += 1
    k = j - n * (n + 1) // 2 - 1          # position within radial order n
    mabs = 2 * ((k + 1) // 2) if n % 2 == 0 else 2 * (k // 2) + 1
    if mabs == 0:
        return n, 0
    return n, (mabs if j % 2 == 0 else -mabs)


def zernike_radial(n: int, m: int, rho: np.ndarray) -> np.ndarray:
    """R_n^|m|(rho) by the explicit factorial sum."""
    m = abs(m)
    out = np.zeros_like(rho, dtype=np.float64)
    for s in range((n - m) // 2 + 1):
        coef = ((-1) ** s * math.factorial(n - s)
                / (math.factorial(s) * math.factorial((n + m) // 2 - s)
                   * math.factorial((n - m) // 2 - s)))
        out += coef * rho ** (n - 2 * s)
    return out


def zernike(j: int, rho: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Noll-normalised Zernike Z_j (unit RMS over the unit disc)."""
    n, m = noll_to_nm(j)
    Rnm = zernike_radial(n, m, rho)
    if m == 0:
        return math.sqrt(n + 1) * Rnm
    ang = np.cos(m * theta) if m > 0 else np.sin(-m * theta)
    return math.sqrt(2 * (n + 1)) * Rnm * ang


def pupil_polar(Np: int) -> tuple[np.ndarray, np.ndarray]:
    """rho (1 at the pupil edge) and theta (from axis 0) at pixel centres."""
    t = (np.arange(Np) - (Np - 1) / 2.0) / (Np / 2.0)
    X, Y = np.meshgrid(t, t, indexing="ij")
    return np.hypot(X, Y), np.arctan2(Y, X)


def zernike_raw(Np: int, obs: float, n_modes: int) -> np.ndarray:
    """Raw Zernikes j = 2..n_modes+1 on the mask pixels (row-major), (n_pix, n_modes)."""
    mask = pupil_mask(Np, obs)
    rho, th = pupil_polar(Np)
    rho, th = rho[mask], th[mask]
    return np.stack([zernike(j, rho, th) for j in range(2, n_modes + 2)], axis=1)


def orthonormalise(Z: np.ndarray) -> np.ndarray:
    """QR in column order, signs so that diag(R) > 0, scaled to unit RMS per column."""
    Q, Rm = np.linalg.qr(Z)
    sgn = np.sign(np.diag(Rm))
    sgn[sgn == 0] = 1.0
    return Q * sgn[None, :] * math.sqrt(Z.shape[0])


def modal_basis(Np: int, obs: float, n_modes: int) -> np.ndarray:
    """DM modal basis M (n_pix, n_modes): 1 unit of coefficient = 1 nm RMS."""
    return orthonormalise(zernike_raw(Np, obs, n_modes))


def basis_to_grid(M: np.ndarray, c: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """DM OPD on the Np x Np grid for modal coefficients c (zero outside the mask)."""
    out = np.zeros(mask.shape)
    out[mask] = M @ c
    return out


def interaction_matrix(measure, M: np.ndarray, mask: np.ndarray, amp_nm: float = 10.0) -> np.ndarray:
    """Push-pull IM: column m = (s(+a M_m) - s(-a M_m)) / (2a); measure(opd) -> slopes."""
    cols = []
    for m in range(M.shape[1]):
        e = np.zeros(M.shape[1])
        e[m] = amp_nm
        sp = measure(basis_to_grid(M, e, mask))
        sm = measure(basis_to_grid(M, -e, mask))
        cols.append((sp - sm) / (2.0 * amp_nm))
    return np.stack(cols, axis=1)


def pseudo_inverse(IM: np.ndarray, rcond: float = 1e-3) -> np.ndarray:
    """R = V diag(1/s) U^T over singular values s >= rcond * s_max (FP64 SVD)."""
    U, s, Vt = np.linalg.svd(IM, full_matrices=False)
    keep = s >= rcond * s[0]
    return (Vt[keep].T / s[keep][None, :]) @ U[:, keep].T


def modal_covariance(M: np.ndarray, mask: np.ndarray, dx: float, r0: float, L0: float,
                     pad: int = 2) -> np.ndarray:
    """Covariance [rad^2 at 500 nm] of the modal coefficients a = (1/n_pix) M^T phi of
    a stationary phase phi with the von Karman PSD (Kolmogorov for L0 = inf):

        C_ij = (1/n_pix^2) sum_f PSD(f) conj(Mhat_i(f)) Mhat_j(f) df^2,
        Mhat_i(f) = sum_x m_i(x) exp(-2 pi i f . x),

    over the frequencies of a (pad Np)^2 zero-padded discrete transform, df = 1 /
    (pad Np dx); for L0 = inf the f = 0 term (infinite PSD) is left out. The
    reading of the KL basis of the 240 px and ELT workloads (the paper names KL
    modes without defining them)."""
    Np = mask.shape[0]
    P = pad * Np
    n = int(mask.sum())
    f = np.fft.fftfreq(P, d=dx)
    fm = np.sqrt(f[:, None] ** 2 + f[None, :] ** 2)
    with np.errstate(divide="ignore"):
        psd = von_karman_psd(fm, r0, L0)
    if math.isinf(L0):
        psd[0, 0] = 0.0
    w = psd.ravel() * (1.0 / (P * dx)) ** 2
    F = np.empty((M.shape[1], P * P), dtype=np.complex128)
    for i in range(M.shape[1]):
        g = np.zeros((P, P))
        g[:Np, :Np][mask] = M[:, i]
        F[i] = np.fft.fft2(g).ravel()
    return ((F.conj() * w) @ F.T).real / (n * n)


def kl_basis(M: np.ndarray, C: np.ndarray):
    """Karhunen-Loeve modes within the span of the orthonormal basis M: M U with
    C = U diag(w) U^T, w decreasing (the coefficient variances). Sign: each mode
    has a positive inner product with sign_pattern (a fixed pattern without the
    pupil's symmetries), a convention independent of the signs of M. Returns
    (M U, w); M's rows are the pupil pixels of `mask` in row-major order."""
    w, U = np.linalg.eigh(C)
    order = np.argsort(-w, kind="stable")
    w, U = w[order], U[:, order]
    K = M @ U
    return K * np.sign(sign_pattern(M.shape[0]) @ K), w


def sign_pattern(n_pix: int) -> np.ndarray:
    """cos(0.73 p + 0.11 + 1.37 sin(0.29 p)) over the pixel list index p."""
    p = np.arange(n_pix, dtype=np.float64)
    return np.cos(0.73 * p + 0.11 + 1.37 * np.sin(0.29 * p))
