"""One-off setup of the loop (not timed per step), host FP64.

The paper's example needs three calibrations before a run (Sec. Example): the
pupil sub-aperture indices, the slope reference vector and the reconstruction
matrix; the DM (Table 1 ``DM``: type 'zernike', nmodes, obsratio) and the
atmosphere (Table 1 ``atmo``/``seeing``) are built from parameters. This module:

  * von Karman phase screens by the FFT method (white noise is an input);
  * the Zernike modal basis in Noll order, orthonormalised on the pupil pixels;
  * the slope reference (a flat wavefront measured by the GPU pyramid);
  * the Zernike basis for large mode counts by Cholesky QR with FP64 products on the
    GPU (the push-pull interaction matrix and its FP64 pseudo-inverse run on the GPU,
    SCAOSystem.calibrate_reconstructor).

Per-step work never runs here: the loop runs in libpas.so's kernels.
"""
from __future__ import annotations

import math

import numpy as np

R0_REF_NM = 500.0
# The KL basis diagonalises the modal covariance built from every mode's spectrum on
# a padded lattice (host FP64): practical up to about this many modes. Larger bases
# use the orthonormal Zernike basis of the same span (zernike_basis_gpu).
KL_MAX_MODES = 1000
# Above this many modes the host Gram-Schmidt gives way to Cholesky QR on the GPU.
HOST_GS_MAX_MODES = 400


def _psd_scale() -> float:
    g = math.gamma
    return (g(11.0 / 6.0) ** 2 / (2.0 * math.pi ** (11.0 / 3.0))) * (24.0 * g(6.0 / 5.0) / 5.0) ** (5.0 / 6.0)


def fft_phase_screen_nm(S: int, pitch_m: float, r0_m: float, L0_m: float, noise: np.ndarray) -> np.ndarray:
    """Periodic S x S von Karman OPD screen [nm], FP64: Re of the inverse DFT of
    noise * sqrt(PSD) * df over the FFT frequency lattice, zero mean."""
    df = 1.0 / (S * pitch_m)
    k = np.fft.fftfreq(S) * S * df                       # cycles / m on the FFT lattice
    f2 = np.add.outer(k * k, k * k)
    f2[0, 0] = 1.0
    outer = 0.0 if math.isinf(L0_m) else (1.0 / L0_m) ** 2
    amp = np.sqrt(_psd_scale() * r0_m ** (-5.0 / 3.0) * (f2 + outer) ** (-11.0 / 6.0)) * df
    amp[0, 0] = 0.0
    field = np.fft.ifft2(noise * amp) * (S * S)
    return field.real * (R0_REF_NM / (2.0 * math.pi))


def layer_screens(cfg, noises) -> np.ndarray:
    """float32 (L, S, S) OPD screens [nm] with the Cn2 fractions applied."""
    out = np.empty((len(cfg.layers), cfg.S, cfg.S), dtype=np.float32)
    for l, (ly, w) in enumerate(zip(cfg.layers, noises)):
        out[l] = fft_phase_screen_nm(cfg.S, cfg.dx, cfg.r0_m * ly.fraction ** -0.6, cfg.L0_m, w)
    return out


# ----------------------------------------------------------------- modal basis

def noll_nm(j: int):
    """Noll index -> (n, m) by enumerating each radial order's azimuthal orders
    (|m| ascending, m != 0 twice); even j carries cos (m > 0), odd j sin."""
    count, n = 0, 0
    while True:
        for mabs in range(n % 2, n + 1, 2):
            for _ in range(1 if mabs == 0 else 2):
                count += 1
                if count == j:
                    return n, (0 if mabs == 0 else (mabs if j % 2 == 0 else -mabs))
        n += 1


def radial_jacobi(n: int, m: int, rho: np.ndarray) -> np.ndarray:
    """R_n^m(rho) = (-1)^((n-m)/2) rho^m P_((n-m)/2)^(m,0)(1 - 2 rho^2)."""
    from scipy.special import eval_jacobi
    k = (n - m) // 2
    return (-1) ** k * rho ** m * eval_jacobi(k, m, 0, 1.0 - 2.0 * rho * rho)


def zernike_basis(Np: int, pupil_flat_idx: np.ndarray, n_modes: int) -> np.ndarray:
    """(n_pix, n_modes) float64, Noll j = 2..n_modes+1, orthonormalised on the
    pupil pixels (modified Gram-Schmidt twice, column order kept) and scaled to
    1 nm RMS per unit coefficient."""
    i, jj = np.divmod(pupil_flat_idx.astype(np.int64), Np)
    x = (i - (Np - 1) / 2.0) / (Np / 2.0)
    y = (jj - (Np - 1) / 2.0) / (Np / 2.0)
    rho = np.hypot(x, y)
    th = np.arctan2(y, x)
    Z = np.empty((rho.size, n_modes))
    for c, j in enumerate(range(2, n_modes + 2)):
        n, m = noll_nm(j)
        r = radial_jacobi(n, abs(m), rho)
        if m == 0:
            Z[:, c] = math.sqrt(n + 1) * r
        elif m > 0:
            Z[:, c] = math.sqrt(2 * (n + 1)) * r * np.cos(m * th)
        else:
            Z[:, c] = math.sqrt(2 * (n + 1)) * r * np.sin(-m * th)
    npix = Z.shape[0]
    Q = Z.copy()
    for _ in range(2):
        for c in range(n_modes):
            v = Q[:, c]
            if c:
                v -= Q[:, :c] @ (Q[:, :c].T @ v)
            Q[:, c] = v / np.linalg.norm(v)
    # sign convention: positive overlap with the raw polynomial
    sgn = np.sign(np.einsum("pc,pc->c", Q, Z))
    sgn[sgn == 0] = 1.0
    return Q * sgn * math.sqrt(npix)


def zernike_raw(Np: int, pupil_flat_idx: np.ndarray, n_modes: int) -> np.ndarray:
    """(n_pix, n_modes) float64 Zernike polynomials Noll j = 2..n_modes+1 at the pupil
    pixel centres (unit RMS on the full disc), the radial parts by the three-term
    recurrence of the Jacobi polynomials P_k^(m,0) in k (DLMF 18.9.1), one azimuthal
    order at a time for all pixels: R_(m+2k)^m(rho) = (-1)^k rho^m P_k^(m,0)(1 - 2 rho^2)."""
    i, jj = np.divmod(pupil_flat_idx.astype(np.int64), Np)
    x = (i - (Np - 1) / 2.0) / (Np / 2.0)
    y = (jj - (Np - 1) / 2.0) / (Np / 2.0)
    rho = np.hypot(x, y)
    th = np.arctan2(y, x)
    t = 1.0 - 2.0 * rho * rho
    nm = [noll_nm(j) for j in range(2, n_modes + 2)]
    need = {}
    for c, (n, m) in enumerate(nm):
        need.setdefault(abs(m), []).append((n, m, c))
    Z = np.empty((rho.size, n_modes))
    for a, items in need.items():
        kmax = max((n - a) // 2 for n, _, _ in items)
        rho_a = rho ** a
        P_prev, P = None, np.ones_like(t)
        polys = [P]
        for k in range(1, kmax + 1):
            if k == 1:
                P_new = (a + 1) + (a + 2) * (t - 1.0) / 2.0
            else:
                s2 = 2 * k + a
                c0 = 2.0 * k * (k + a) * (s2 - 2)
                c1 = (s2 - 1) * ((s2) * (s2 - 2) * t + a * a)
                c2 = 2.0 * (k + a - 1) * (k - 1) * s2
                P_new = (c1 * P - c2 * P_prev) / c0
            P_prev, P = P, P_new
            polys.append(P)
        for n, m, c in items:
            k = (n - a) // 2
            r = (-1) ** k * rho_a * polys[k]
            if m == 0:
                Z[:, c] = math.sqrt(n + 1) * r
            elif m > 0:
                Z[:, c] = math.sqrt(2 * (n + 1)) * r * np.cos(m * th)
            else:
                Z[:, c] = math.sqrt(2 * (n + 1)) * r * np.sin(-m * th)
    return Z


def zernike_basis_gpu(ctx, Np: int, pupil_flat_idx: np.ndarray, n_modes: int, passes: int = 2) -> np.ndarray:
    """The Zernike basis of zernike_basis (Noll order, orthonormal on the pupil pixels,
    1 nm RMS per unit coefficient) for large mode counts: Cholesky QR repeated
    `passes` times, Q = Z L^-T with L L^T = Z^T Z, the Gram matrices and the products
    in FP64 on the GPU (pas_gemm_f64), the n x n Cholesky factor on the host. Column
    order is kept (R = L^T upper triangular with a positive diagonal), so Q is the
    Gram-Schmidt basis of the same columns. Returns float64 (n_pix, n_modes)."""
    import torch
    from . import pas as P
    Z = zernike_raw(Np, pupil_flat_idx, n_modes)
    m, n = Z.shape
    dev = torch.device("cuda")
    Zd = torch.as_tensor(np.ascontiguousarray(Z.T)).to(dev)     # column a of Z at Zd[a]
    raw = Zd.clone()
    del Z
    G = torch.empty(n, n, device=dev, dtype=torch.float64)
    for _ in range(passes):
        # G[a][b] = sum_k Z[k, a] Z[k, b]
        P.pas_gemm_f64(ctx, Zd, m, 1, Zd, m, 1, None, n, n, m, G, n)
        torch.cuda.synchronize()
        L = np.linalg.cholesky(0.5 * (G.cpu().numpy() + G.cpu().numpy().T))
        T = np.linalg.solve(L, np.eye(n)).T                   # L^-T (upper triangular)
        Td = torch.as_tensor(np.ascontiguousarray(T)).to(dev)
        Q = torch.empty_like(Zd)
        # Q[b][k] = sum_a T[a][b] Z[k, a]
        P.pas_gemm_f64(ctx, Td, 1, n, Zd, 1, m, None, n, m, n, Q, m)
        torch.cuda.synchronize()
        Zd = Q
    # sign convention of zernike_basis: positive overlap with the raw polynomial
    sgn = torch.sign((Zd * raw).sum(dim=1))
    sgn[sgn == 0] = 1.0
    Zd *= (sgn * math.sqrt(m))[:, None]
    return Zd.t().cpu().numpy()


def modal_covariance(basis: np.ndarray, pix: np.ndarray, Np: int, pitch_m: float, r0_m: float, L0_m: float,
                     pad: int = 2, chunk: int = 64) -> np.ndarray:
    """Covariance [rad^2 at the r0 wavelength] of the coefficients a = (1/n) B^T phi
    of von Karman turbulence on the basis B (n pupil pixels x modes):
    (1/n^2) sum over the (pad Np)^2 frequency lattice of PSD(f) df^2 Re(conj(Bhat_i) Bhat_j).
    Real mode maps have Hermitian spectra, so only the half spectrum of rfft2 is
    formed, each column other than 0 and the Nyquist one counted twice, and the
    complex sum splits into two real matrix products."""
    P = pad * Np
    n, nm = basis.shape
    df = 1.0 / (P * pitch_m)
    fy = np.fft.fftfreq(P, d=pitch_m)
    fx = np.fft.rfftfreq(P, d=pitch_m)
    f2 = np.add.outer(fy * fy, fx * fx)
    outer = 0.0 if math.isinf(L0_m) else (1.0 / L0_m) ** 2
    with np.errstate(divide="ignore"):
        psd = _psd_scale() * r0_m ** (-5.0 / 3.0) * (f2 + outer) ** (-11.0 / 6.0)
    if math.isinf(L0_m):
        psd[0, 0] = 0.0
    mult = np.full(fx.size, 2.0)
    mult[0] = 1.0
    if P % 2 == 0:
        mult[-1] = 1.0
    w = (psd * mult[None, :] * df * df).ravel()
    rows, cols = np.divmod(np.asarray(pix, dtype=np.int64), Np)
    re = np.empty((nm, w.size))
    im = np.empty((nm, w.size))
    for c0 in range(0, nm, chunk):
        c1 = min(nm, c0 + chunk)
        g = np.zeros((c1 - c0, P, P))
        g[:, rows, cols] = basis[:, c0:c1].T
        spec = np.fft.rfft2(g).reshape(c1 - c0, -1)
        re[c0:c1] = spec.real
        im[c0:c1] = spec.imag
    C = (re * w) @ re.T + (im * w) @ im.T
    return C / (float(n) * n)


_KL_CACHE: dict = {}


def kl_basis(Np: int, pix: np.ndarray, n_modes: int, pitch_m: float, r0_m: float, L0_m: float,
             pad: int = 2) -> np.ndarray:
    """Karhunen-Loeve modes of von Karman turbulence within the span of the first
    n_modes Zernike modes: eigenvectors of their coefficient covariance, variances
    decreasing, each mode with a positive inner product with the fixed pattern
    cos(0.73 p + 0.11 + 1.37 sin(0.29 p)) over the pixel index p (a sign that does
    not depend on the Zernike signs); float64 (n pixels x n_modes), orthonormal
    (B^T B = n I). Cached per geometry."""
    key = (Np, hash(np.asarray(pix).tobytes()), n_modes, pitch_m, r0_m, L0_m, pad)
    if key not in _KL_CACHE:
        Z = zernike_basis(Np, pix, n_modes)
        C = modal_covariance(Z, pix, Np, pitch_m, r0_m, L0_m, pad)
        w, U = np.linalg.eigh(0.5 * (C + C.T))
        U = U[:, np.argsort(-w, kind="stable")]
        K = Z @ U
        q = np.arange(K.shape[0], dtype=np.float64)
        K *= np.sign(np.cos(0.73 * q + 0.11 + 1.37 * np.sin(0.29 * q)) @ K)
        _KL_CACHE[key] = K
    return _KL_CACHE[key]


def wind_shift_px(cfg) -> np.ndarray:
    """(L, 2) float64: each layer's screen shift per loop step in pixels along axis 0
    and axis 1, v dt / dx rotated by the wind direction (counter-clockwise from axis
    0; Table 1 wind_speed / wind_direction, main time_step)."""
    out = np.empty((len(cfg.layers), 2))
    for l, ly in enumerate(cfg.layers):
        px_per_step = ly.wind_mps * cfg.dt_s * cfg.Np / cfg.D
        a = math.radians(ly.wind_dir_deg)
        out[l] = (px_per_step * math.cos(a), px_per_step * math.sin(a))
    return out


def detector_photons(cfg) -> float:
    """Photons per detector frame for the guide star's magnitude (Table 1
    wfs_source.magnitude, detector bandw / quantum_eff, time step): zero point x
    10^(-m/2.5) x (pi/4) D^2 (1 - obs^2) x bandwidth x QE x dt; 0 when noiseless."""
    if cfg.magnitude is None:
        return 0.0
    area_m2 = math.pi * (cfg.D / 2.0) ** 2 - math.pi * (cfg.obs * cfg.D / 2.0) ** 2
    return (cfg.zero_point_ph_s_m2_nm * 10.0 ** (-cfg.magnitude / 2.5) * area_m2 * cfg.bandwidth_nm * cfg.qe
            * cfg.dt_s)


def footprint_offsets_px(heights_m, rho_arcsec: float, phi_deg: float, dx: float):
    """Per-layer footprint offsets (ox, oy) in screen pixels of a natural guide star
    off axis at (rho arcsec, phi degrees counter-clockwise from axis 0): layer h is
    crossed at h * theta from the on-axis footprint (Table 1 wfs_source
    polar_coordinate; a source at infinity, no footprint scaling)."""
    theta = math.radians(rho_arcsec / 3600.0)
    phi = math.radians(phi_deg)
    return [(h * theta * math.cos(phi) / dx, h * theta * math.sin(phi) / dx) for h in heights_m]


def footprint_scales(heights_m, H_m: float):
    """Per-layer footprint scales 1 - h/H of a source at height H (a laser guide
    star): the cone from the pupil to the source crosses layer h on a disc shrunk by
    that factor (sources at finite distance, abstract; LGS SCAO systems, Sec.
    History/Reference works)."""
    if not H_m > max(heights_m):
        raise ValueError("the source must lie above every layer")
    return [1.0 - h / H_m for h in heights_m]


def disc_source(diameter_lod: float, n_across: int):
    """A uniform disc of angular diameter `diameter_lod` lambda/D as point sources on an
    n_across x n_across grid of spacing diameter / n_across (those inside the disc;
    equal intensities): (ex, ey) for pas_pyr_create_extended (extended reference
    sources, Sec. History/Reference works)."""
    h = diameter_lod / n_across
    c = (np.arange(n_across) - (n_across - 1) / 2.0) * h
    X, Y = np.meshgrid(c, c, indexing="ij")
    inside = X ** 2 + Y ** 2 <= (diameter_lod / 2.0) ** 2 + 1e-12
    return X[inside].copy(), Y[inside].copy()
