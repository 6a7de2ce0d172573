"""Oracle optics: pupil stop, centred DFT, modulated four-face pyramid, detector, slopes.

Paper passages: the pyramid object and its parameters (Table 1, ``pyramid``:
pup_diam, pup_dist, mod_amp, output_resolution, wavelengthInNm), the pupil stop
(Table 1 ``pupil_stop``, ``DM.obsratio``), the detector (Table 1 ``detector``), the
slope computer with pupil indices and slope reference (Table 1 ``slopec``; Table 3
pupil calibration) and the GPU area "pyramid propagation from wavefront to detector
plane" (Sec. GPU acceleration). The paper gives no formula for any of them; the
readings below are the textbook Fourier-optics model.

Conventions (readings):
  * axis 0 = x (rows), axis 1 = y (columns); pixel centres x~ = i - (n-1)/2;
  * the centred unitary DFT  X(u) = N^-1/2 sum_x x(x) exp(-2 pi i x~ u~ / N)
    with half-integer centred coordinates in both planes;
  * pyramid mask P(u, v) = exp(i 2 pi delta (|u~| + |v~|) / N), delta = N/4, so
    the face with positive frequencies images to the low half of each axis;
  * modulation point k at angle theta_k = 2 pi k / K from axis 0, radius R lambda/D,
    tilt psi_k = 2 pi R (X cos theta_k + Y sin theta_k), X = x~/Np;
  * intensity I = (1/K) sum_k |g_k|^2 summed over the whole N x N grid into b x b
    blocks, the four pupil images being the four grid quadrants.
"""
from __future__ import annotations

import math

import numpy as np


# --------------------------------------------------------------------------- pupil

def obstruction_threshold(Np: int, obs: float) -> int:
    """Smallest integer T with T >= (obs*Np)^2 - 1e-9: pixels with
    (2i-Np+1)^2 + (2j-Np+1)^2 >= T are outside the central obstruction.
    The 1e-9 slack makes obs*Np = 24.000000000000004 count as 24."""
    t = obs * Np
    return int(math.ceil(t * t - 1e-9))


def pupil_mask(Np: int, obs: float) -> np.ndarray:
    """Annular pupil stop on an Np x Np grid (Table 1 pupil_stop.obs_diam).

    Pixel (i, j) is inside iff d2 = (2i-Np+1)^2 + (2j-Np+1)^2 <= Np^2 and
    d2 >= obstruction_threshold(Np, obs): the outer diameter equals Np pixels and
    the test is done in integers."""
    i = np.arange(Np, dtype=np.int64)
    a = (2 * i - Np + 1) ** 2
    d2 = a[:, None] + a[None, :]
    return (d2 <= Np * Np) & (d2 >= obstruction_threshold(Np, obs))


def pixel_coords(Np: int) -> tuple[np.ndarray, np.ndarray]:
    """Pupil-normalised pixel-centre coordinates X, Y in (-1/2, 1/2) (D = 1)."""
    x = (np.arange(Np) - (Np - 1) / 2.0) / Np
    return np.meshgrid(x, x, indexing="ij")


def embed(field: np.ndarray, N: int) -> np.ndarray:
    """Centre an Np x Np field in an N x N zero grid (offset (N-Np)/2)."""
    Np = field.shape[0]
    off = (N - Np) // 2
    out = np.zeros((N, N), dtype=np.complex128)
    out[off:off + Np, off:off + Np] = field
    return out


# --------------------------------------------------------------------------- DFT

def centred_dft_matrix(N: int) -> np.ndarray:
    """W[u, x] = N^-1/2 exp(-2 pi i (x - c)(u - c) / N), c = (N-1)/2. Symmetric, unitary."""
    c = (N - 1) / 2.0
    t = np.arange(N) - c
    return np.exp(-2j * np.pi * np.outer(t, t) / N) / math.sqrt(N)


def cdft2(E: np.ndarray) -> np.ndarray:
    """Centred unitary 2-D DFT as the matrix product W E W^T (W = W^T)."""
    W = centred_dft_matrix(E.shape[0])
    return W @ E @ W


def icdft2(G: np.ndarray) -> np.ndarray:
    """Inverse of cdft2: W^H G W^H (W unitary and symmetric)."""
    Wh = np.conj(centred_dft_matrix(G.shape[0]))
    return Wh @ G @ Wh


def _ramp(N: int) -> np.ndarray:
    c = (N - 1) / 2.0
    return np.exp(2j * np.pi * c * np.arange(N) / N)


def cdft2_fft(E: np.ndarray) -> np.ndarray:
    """cdft2 through numpy.fft: (x-c)(u-c) = xu - cx - cu + c^2 gives a pre-ramp,
    a post-ramp and a constant phase (once per axis) around the standard DFT."""
    N = E.shape[0]
    r = _ramp(N)
    const = np.exp(-2j * np.pi * 2.0 * ((N - 1) / 2.0) ** 2 / N) / N
    pre = E * np.outer(r, r)
    return const * np.fft.fft2(pre) * np.outer(r, r)


def icdft2_fft(G: np.ndarray) -> np.ndarray:
    N = G.shape[0]
    rc = np.conj(_ramp(N))
    const = np.exp(2j * np.pi * 2.0 * ((N - 1) / 2.0) ** 2 / N) * N
    pre = G * np.outer(rc, rc)
    return const * np.fft.ifft2(pre) * np.outer(rc, rc)


# --------------------------------------------------------------------------- pyramid

def pyramid_mask(N: int, delta: float) -> np.ndarray:
    """Four-face pyramid phase mask P(u,v) = exp(i 2 pi delta (|u~| + |v~|) / N)."""
    t = np.abs(np.arange(N) - (N - 1) / 2.0)
    return np.exp(2j * np.pi * delta * (t[:, None] + t[None, :]) / N)


def modulation_angles(K: int) -> np.ndarray:
    """theta_k = 2 pi k / K, equal weights (Table 1 pyramid.mod_amp)."""
    return 2.0 * np.pi * np.arange(K) / K


def tilt_phase(Np: int, R: float, theta: float) -> np.ndarray:
    """Modulation tilt psi = 2 pi R (X cos theta + Y sin theta) [rad], R in lambda/D."""
    X, Y = pixel_coords(Np)
    return 2.0 * np.pi * R * (X * math.cos(theta) + Y * math.sin(theta))


def pwfs_intensity(opd_nm: np.ndarray, wavelength_nm: float, obs: float, N: int, K: int,
                   R: float, delta: float | None = None, use_fft: bool = True,
                   amplitude: np.ndarray | None = None) -> np.ndarray:
    """Modulated pyramid intensity on the N x N pupil-image plane.

    For every modulation point k: pupil field A exp(i(2 pi opd/lambda + psi_k)),
    centred in the N grid, centred DFT to the focal plane, times the pyramid mask,
    inverse centred DFT back to the pupil plane, |.|^2; averaged over the K points.
    ``use_fft`` selects numpy.fft with ramps instead of the explicit matrix
    product (both are the same transform; a test checks it)."""
    Np = opd_nm.shape[0]
    delta = N / 4.0 if delta is None else delta
    A = pupil_mask(Np, obs).astype(np.float64) if amplitude is None else amplitude
    phi = 2.0 * np.pi * np.asarray(opd_nm, dtype=np.float64) / wavelength_nm
    P = pyramid_mask(N, delta)
    fwd, inv = (cdft2_fft, icdft2_fft) if use_fft else (cdft2, icdft2)
    I = np.zeros((N, N))
    for th in modulation_angles(K):
        E = embed(A * np.exp(1j * (phi + tilt_phase(Np, R, th))), N)
        g = inv(fwd(E) * P)
        I += np.abs(g) ** 2
    return I / K


def pwfs_intensity_extended(opd_nm: np.ndarray, wavelength_nm: float, obs: float, N: int, K: int, R: float,
                            ex, ey, w=None, delta: float | None = None, use_fft: bool = True) -> np.ndarray:
    """Modulated pyramid intensity of an extended incoherent source (Sec. History/
    Reference works, extended reference sources; Sec. Conclusions, their cost at ELT
    scale): sum_p w_p I_p with I_p the modulated intensity of point source p, whose
    wavefront carries the tilt 2 pi (ex_p X + ey_p Y) of its offset (ex_p, ey_p)
    lambda/D from the source centre (the modulation's own tilt convention); the
    weights are normalised to sum 1 (None: equal)."""
    ex = np.atleast_1d(np.asarray(ex, dtype=np.float64))
    ey = np.atleast_1d(np.asarray(ey, dtype=np.float64))
    w = np.ones(ex.size) if w is None else np.atleast_1d(np.asarray(w, dtype=np.float64))
    w = w / w.sum()
    X, Y = pixel_coords(opd_nm.shape[0])
    I = np.zeros((N, N))
    for xp, yp, wp in zip(ex, ey, w):
        opd_p = np.asarray(opd_nm, dtype=np.float64) + wavelength_nm * (xp * X + yp * Y)
        I += wp * pwfs_intensity(opd_p, wavelength_nm, obs, N, K, R, delta, use_fft)
    return I


# --------------------------------------------------------------------------- detector

def bin_detector(I: np.ndarray, b: int) -> np.ndarray:
    """Detector pixel = sum of its b x b block of the N x N intensity (Table 1
    pyramid.output_resolution / detector.size)."""
    N = I.shape[0]
    n = N // b
    assert n * b == N
    return I.reshape(n, b, n, b).sum(axis=(1, 3))


def overlap_units(n_fine: int, n_coarse: int) -> np.ndarray:
    """O[s, i] = length of fine pixel [i, i+1) inside coarse pixel s (which spans
    [s n_fine / n_coarse, (s+1) n_fine / n_coarse)), in units of 1/n_coarse: an
    integer in [0, n_coarse]. Scaling both intervals by n_coarse makes the ends
    integers: [i n_coarse, (i+1) n_coarse) and [s n_fine, (s+1) n_fine)."""
    i = np.arange(n_fine, dtype=np.int64)[None, :]
    s = np.arange(n_coarse, dtype=np.int64)[:, None]
    lo = np.maximum(i * n_coarse, s * n_fine)
    hi = np.minimum((i + 1) * n_coarse, (s + 1) * n_fine)
    return np.maximum(hi - lo, 0)


def rebin(I: np.ndarray, nd: int) -> np.ndarray:
    """Area-weighted rebinning of the N x N intensity onto nd x nd detector pixels of
    side b = N / nd fine pixels, b not necessarily an integer (the detector of the
    batched workload: 20 sub-apertures on 128 pupil pixels, 60 on 320). Each fine
    pixel splits its value among the detector pixels it overlaps in proportion to
    the overlap area, so the frame keeps the total; integer b gives block sums."""
    N = I.shape[0]
    W = overlap_units(N, nd).astype(np.float64) / nd
    return W @ np.asarray(I, dtype=np.float64) @ W.T


def detector_frame(I: np.ndarray, n_sub: int) -> np.ndarray:
    """The (2 n_sub)^2 detector frame of an N x N intensity: block sums when
    N / (2 n_sub) is an integer, area-weighted rebinning otherwise."""
    N = I.shape[0]
    if N % (2 * n_sub) == 0:
        return bin_detector(I, N // (2 * n_sub))
    return rebin(I, 2 * n_sub)


def subaperture_area_units(mask: np.ndarray, n_sub: int) -> np.ndarray:
    """Pupil area inside each sub-aperture in units of 1/n_sub^2 fine pixels
    (integers): A = O mask O^T with O = overlap_units(Np, n_sub)."""
    O = overlap_units(mask.shape[0], n_sub)
    return O @ mask.astype(np.int64) @ O.T


def subaperture_counts(mask: np.ndarray, n_sub: int) -> np.ndarray:
    """Number of pupil pixels in each b x b sub-aperture block (integer b)."""
    Np = mask.shape[0]
    b = Np // n_sub
    assert b * n_sub == Np
    return mask.astype(np.int64).reshape(n_sub, b, n_sub, b).sum(axis=(1, 3))


def valid_subapertures(Np: int, obs: float, n_sub: int) -> np.ndarray:
    """Valid sub-apertures: 2 * (pupil area in the sub-aperture) >= b^2 (geometric
    rule, b = Np / n_sub). In the integer units of subaperture_area_units the rule
    reads 2 A >= Np^2; for integer b it is 2 * (pupil pixels in the block) >= b^2.
    Returns int32 flat indices r*n_sub + c in row-major order (the pupil index data
    of the slope computer, Table 1 slopec.pupdata_tag, Table 3)."""
    A = subaperture_area_units(pupil_mask(Np, obs), n_sub)
    return np.flatnonzero((2 * A).ravel() >= Np * Np).astype(np.int32)


def valid_subapertures_threshold(frame: np.ndarray, n_sub: int, thr: float) -> np.ndarray:
    """Table 3's acquisition rule as a cross-check: threshold the sum of the four
    pupil images of a flat, strongly modulated frame at ``thr`` times its maximum."""
    q = (frame[:n_sub, :n_sub] + frame[:n_sub, n_sub:] + frame[n_sub:, :n_sub]
         + frame[n_sub:, n_sub:])
    return np.flatnonzero(q.ravel() >= thr * q.max()).astype(np.int32)


def quadrant_values(frame: np.ndarray, valid: np.ndarray, n_sub: int):
    """The four detector pixels of each valid sub-aperture: (q00, q01, q10, q11),
    q_ab with a = row half and b = column half of the detector."""
    r = valid // n_sub
    c = valid % n_sub
    return (frame[r, c], frame[r, n_sub + c], frame[n_sub + r, c],
            frame[n_sub + r, n_sub + c])


def pwfs_slopes(frame: np.ndarray, valid: np.ndarray, n_sub: int,
                sn: np.ndarray | None = None, local: bool = False) -> np.ndarray:
    """Normalised pyramid slopes [Sx; Sy] over the valid sub-apertures.

    Sx = (q10 + q11 - q00 - q01) / F   (row halves: axis 0)
    Sy = (q01 + q11 - q00 - q10) / F   (column halves: axis 1)
    F = mean over valid sub-apertures of q00+q01+q10+q11 (global normalisation;
    ``local`` divides by each sub-aperture's own total). The slope reference
    ``sn`` (Table 1 slopec.sn_tag) is subtracted."""
    q00, q01, q10, q11 = quadrant_values(np.asarray(frame, dtype=np.float64), valid, n_sub)
    tot = q00 + q01 + q10 + q11
    F = tot if local else tot.mean()
    s = np.concatenate([(q10 + q11 - q00 - q01) / F, (q01 + q11 - q00 - q10) / F])
    if sn is not None:
        s = s - sn
    return s


def pwfs_measure(opd_nm, cfg, valid=None, sn=None, use_fft=True):
    """opd -> (frame, slopes) for a configuration (noiseless)."""
    I = pwfs_intensity(opd_nm, cfg.wavelength_nm, cfg.obs, cfg.N, cfg.K, cfg.mod_radius,
                       cfg.delta, use_fft=use_fft)
    frame = detector_frame(I, cfg.n_sub)
    if valid is None:
        valid = valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    return frame, pwfs_slopes(frame, valid, cfg.n_sub, sn)
