"""Oracle atmosphere: von Karman phase screens (FFT method) and wind shift.

Paper passages: the atmosphere container and its parameters (Table 1 ``atmo``: L0,
heights, Cn2; ``seeing``; ``wind_speed``; ``wind_direction``), the propagation
object that sums the layers onto the pupil along the source direction (Table 2
``get_atmo_propagation``, ``add_layer_to_layer_list``) and the GPU area "wavefront
propagation through phase screens" (Sec. GPU acceleration). No formula is printed;
the readings are:

  * phase power spectrum Phi(f) = 0.0229 r0^-5/3 (f^2 + L0^-2)^-11/6 [rad^2 m^2 at
    500 nm] (the constant written out exactly below); L0 = inf gives Kolmogorov;
  * FFT method, no subharmonics: phase = Re( sum_f w_f sqrt(Phi(f)) df
    exp(2 pi i f.x) ), w_f = a + i b with a, b unit normals (passed in), f = 0 set
    to zero, df = 1/(S dx); the screen is periodic with pitch dx;
  * layer l of Cn2 fraction f_l has r0_l = r0 f_l^-3/5; OPD [nm] = phase 500/(2 pi);
  * on-axis source: the layer's pupil footprint is the pupil itself, shifted by the
    wind: at step t the pupil pixel (i, j) samples the screen at
    (i - t vx, j - t vy), vx, vy in pixels per step (FP64, no running sum),
    bilinear interpolation with periodic wrap;
  * a natural guide star off axis at polar coordinates (rho arcsec, phi degrees
    counter-clockwise from axis 0; Table 1 wfs_source.polar_coordinate) sees layer l
    at height h_l through a footprint moved by h_l theta: pixel (i, j) samples
    (i + ox_l - t vx, j + oy_l - t vy) with (ox_l, oy_l) = h_l theta (cos phi, sin phi)
    / dx, theta = rho in radians (no footprint scaling: the source is at infinity);
  * a source at finite height H (a laser guide star) sees layer l through a footprint
    shrunk by s_l = 1 - h_l / H about the pupil centre c = (Np - 1) / 2 (the cone
    effect): pixel i samples c + (i - c) s_l + ox_l - t vx (offsets h_l theta as above;
    sources at finite distance: abstract; LGS SCAO systems: Sec. History/Reference works).
"""
from __future__ import annotations

import math

import numpy as np

R0_WAVELENGTH_NM = 500.0


def psd_constant() -> float:
    """(24/5 Gamma(6/5))^(5/6) Gamma(11/6)^2 / (2 pi^(11/3)) = 0.02289..."""
    return ((24.0 / 5.0 * math.gamma(6.0 / 5.0)) ** (5.0 / 6.0) * math.gamma(11.0 / 6.0) ** 2
            / (2.0 * math.pi ** (11.0 / 3.0)))


def von_karman_psd(f: np.ndarray, r0: float, L0: float) -> np.ndarray:
    """Phase PSD [rad^2 m^2] at 500 nm; f in cycles per metre; L0 = inf: Kolmogorov."""
    inv_L0_sq = 0.0 if math.isinf(L0) else 1.0 / (L0 * L0)
    return psd_constant() * r0 ** (-5.0 / 3.0) * (np.asarray(f) ** 2 + inv_L0_sq) ** (-11.0 / 6.0)


def phase_screen_rad(S: int, dx: float, r0: float, L0: float, w: np.ndarray) -> np.ndarray:
    """One periodic S x S phase screen [rad at 500 nm] from complex white noise w."""
    f = np.fft.fftfreq(S, d=dx)
    fmag = np.sqrt(f[:, None] ** 2 + f[None, :] ** 2)
    with np.errstate(divide="ignore"):
        psd = von_karman_psd(fmag, r0, L0)
    psd[0, 0] = 0.0
    df = 1.0 / (S * dx)
    C = w * np.sqrt(psd) * df
    # sum_f C_f exp(2 pi i f x) over the FFT frequency grid = S^2 * ifft2(C)
    return np.real(np.fft.ifft2(C)) * (S * S)


def layer_screens_nm(cfg, noises: list[np.ndarray]) -> np.ndarray:
    """All layers of a configuration as OPD screens [nm], shape (L, S, S)."""
    out = np.empty((len(cfg.layers), cfg.S, cfg.S))
    for l, (ly, w) in enumerate(zip(cfg.layers, noises)):
        r0_l = cfg.r0_m * ly.fraction ** (-3.0 / 5.0)
        out[l] = phase_screen_rad(cfg.S, cfg.dx, r0_l, cfg.L0_m, w) * R0_WAVELENGTH_NM / (2 * math.pi)
    return out


def bilinear_sample(screen: np.ndarray, px: np.ndarray, py: np.ndarray) -> np.ndarray:
    """Bilinear interpolation of a periodic screen at positions (px, py) [pixels]."""
    S = screen.shape[0]
    x0 = np.floor(px)
    y0 = np.floor(py)
    fx = px - x0
    fy = py - y0
    i0 = x0.astype(np.int64) % S
    j0 = y0.astype(np.int64) % S
    i1 = (i0 + 1) % S
    j1 = (j0 + 1) % S
    return ((1 - fx) * (1 - fy) * screen[i0, j0] + fx * (1 - fy) * screen[i1, j0]
            + (1 - fx) * fy * screen[i0, j1] + fx * fy * screen[i1, j1])


def wind_velocity_px(cfg):
    """Per-layer screen displacement per loop step, in screen pixels along (axis 0,
    axis 1): speed * time step / pixel pitch, split by the wind direction measured
    counter-clockwise from axis 0 (Table 1 wind_speed, wind_direction; main
    time_step; the pitch is D / Np)."""
    pitch = cfg.D / cfg.Np
    out = []
    for ly in cfg.layers:
        d = ly.wind_mps * cfg.dt_s / pitch
        ang = ly.wind_dir_deg * math.pi / 180.0
        out.append((d * math.cos(ang), d * math.sin(ang)))
    return out


def layer_offset(step: int, v: float) -> float:
    """Wind displacement after ``step`` steps [px], one FP64 product."""
    return float(step) * v


def footprint_offsets_px(heights_m, rho_arcsec: float, phi_deg: float, dx: float):
    """Per-layer footprint offsets (ox, oy) [px] for a source at infinity in the
    direction (rho arcsec, phi degrees from axis 0)."""
    theta = rho_arcsec * math.pi / (180.0 * 3600.0)
    c, s = math.cos(math.radians(phi_deg)), math.sin(math.radians(phi_deg))
    return [(h * theta * c / dx, h * theta * s / dx) for h in heights_m]


def footprint_scales(heights_m, H_m: float):
    """Per-layer footprint scale 1 - h / H of a source at height H (cone effect)."""
    return [1.0 - h / H_m for h in heights_m]


def atmo_opd(screens_nm: np.ndarray, velocities_px, step: int, Np: int, offsets_px=None,
             scales=None) -> np.ndarray:
    """Sum over layers of the wind-shifted screens on the Np x Np pupil grid [nm],
    each layer's footprint moved by its (ox, oy) offset [px] and shrunk by its scale
    about the pupil centre when given."""
    i = np.arange(Np, dtype=np.float64)
    I, J = np.meshgrid(i, i, indexing="ij")
    c = (Np - 1) / 2.0
    out = np.zeros((Np, Np))
    if offsets_px is None:
        offsets_px = [(0.0, 0.0)] * len(velocities_px)
    if scales is None:
        scales = [1.0] * len(velocities_px)
    for scr, (vx, vy), (ox, oy), sc in zip(screens_nm, velocities_px, offsets_px, scales):
        Ii = I if sc == 1.0 else c + (I - c) * sc
        Jj = J if sc == 1.0 else c + (J - c) * sc
        out += bilinear_sample(scr, Ii + (ox - layer_offset(step, vx)), Jj + (oy - layer_offset(step, vy)))
    return out


# ----------------------------------------------------------------- statistics (pins)

def structure_function_kolmogorov(r: np.ndarray, r0: float) -> np.ndarray:
    """Textbook D(r) = 6.88 (r/r0)^(5/3) [rad^2]."""
    return 6.88 * (np.asarray(r) / r0) ** (5.0 / 3.0)


def structure_function_von_karman(r: np.ndarray, r0: float, L0: float) -> np.ndarray:
    """Closed form of D(r) = 2 (B(0) - B(r)) for the von Karman spectrum above.

    B(r) = 2 pi int_0^inf Phi(f) J0(2 pi f r) f df evaluates (Gradshteyn-Ryzhik
    6.565.4 with mu = 5/6) to 2 pi c / (2^(5/6) Gamma(11/6)) (L0/r0)^(5/3)
    x^(5/6) K_5/6(x), x = 2 pi r / L0, so that
    D(r) = 2 pi c Gamma(5/6)/Gamma(11/6) (L0/r0)^(5/3) [1 - 2^(1/6)/Gamma(5/6) x^(5/6) K_5/6(x)]
    (prefactor 0.1727 (L0/r0)^(5/3))."""
    from scipy.special import kv
    r = np.asarray(r, dtype=np.float64)
    c = psd_constant()
    g56 = math.gamma(5.0 / 6.0)
    two_b0 = 2.0 * math.pi * c * g56 / math.gamma(11.0 / 6.0)
    x = 2.0 * math.pi * r / L0
    xs = np.maximum(x, 1e-300)
    xk = np.where(x > 0, xs ** (5.0 / 6.0) * kv(5.0 / 6.0, xs), 2.0 ** (-1.0 / 6.0) * g56)
    return two_b0 * (L0 / r0) ** (5.0 / 3.0) * (1.0 - 2.0 ** (1.0 / 6.0) / g56 * xk)


def structure_function_expected_fft(S: int, dx: float, r0: float, L0: float,
                                    r_px: np.ndarray) -> np.ndarray:
    """Expected D(r) of FFT screens (no subharmonics) along axis 0 at lags r_px:
    sum over the FFT frequency grid of Phi df^2 2 (1 - cos(2 pi fx r))."""
    f = np.fft.fftfreq(S, d=dx)
    FX = f[:, None] + 0 * f[None, :]
    fmag = np.sqrt(f[:, None] ** 2 + f[None, :] ** 2)
    with np.errstate(divide="ignore"):
        psd = von_karman_psd(fmag, r0, L0)
    psd[0, 0] = 0.0
    df = 1.0 / (S * dx)
    return np.array([np.sum(psd * df * df * 2 * (1 - np.cos(2 * np.pi * FX * r * dx)))
                     for r in np.atleast_1d(r_px)])
