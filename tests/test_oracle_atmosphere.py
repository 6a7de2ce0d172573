"""Pins of the oracle's atmosphere: PSD constant, structure functions, wind shift."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import j0

from oracle import atmosphere as at
from synth import get_config, tiny_config
from synth.inputs import screen_white_noise


def test_psd_constant_matches_textbook_value():
    # the printed textbook constant is 0.023 (0.0229 to three figures)
    assert abs(at.psd_constant() - 0.0229) < 1e-4


@pytest.mark.parametrize("r", [0.05, 0.3, 1.0, 4.0, 20.0])
def test_von_karman_closed_form_against_quadrature(r):
    r0, L0 = 0.12, 25.0
    f = lambda x: at.von_karman_psd(x, r0, L0) * (1 - j0(2 * math.pi * x * r)) * x * 4 * math.pi
    q = quad(f, 0, np.inf, limit=4000)[0]
    assert abs(at.structure_function_von_karman(r, r0, L0) - q) / q < 1e-6


def test_kolmogorov_psd_gives_6p88_law():
    """Quadrature of the L0 = inf spectrum: D(r) = 6.88 (r/r0)^(5/3) (the exact
    prefactor 2 (24/5 Gamma(6/5))^(5/6) = 6.8839 is printed rounded to 6.88)."""
    r0 = 0.1
    for r in (0.01, 0.1, 1.0):
        f = lambda x: at.von_karman_psd(x, r0, math.inf) * (1 - j0(2 * math.pi * x * r)) * x * 4 * math.pi
        q = sum(quad(f, a, b, limit=4000)[0] for a, b in ((0, 1 / r), (1 / r, 100 / r), (100 / r, np.inf)))
        assert abs(q / at.structure_function_kolmogorov(r, r0) - 1) < 1e-3
    # and the von Karman closed form approaches it for r << L0
    assert abs(at.structure_function_von_karman(1e-3, r0, 1e4) / at.structure_function_kolmogorov(1e-3, r0) - 1) < 0.02


def _empirical_D(screen, lags):
    return np.array([np.mean((np.roll(screen, -r, axis=0) - screen) ** 2) for r in lags])


def test_fft_screen_statistics_match_expectation():
    """Monte-Carlo D(r) of FFT screens equals the exact discrete expectation
    (normalisation, df, the factor of Re, the frequency grid)."""
    S, dx, r0, L0 = 128, 0.05, 0.1, 25.0
    lags = np.array([1, 2, 4, 8, 16])
    acc = np.zeros(lags.size)
    n = 48
    for seed in range(n):
        acc += _empirical_D(at.phase_screen_rad(S, dx, r0, L0, screen_white_noise(S, 500 + seed)), lags)
    emp = acc / n
    exp = at.structure_function_expected_fft(S, dx, r0, L0, lags)
    assert np.all(np.abs(emp / exp - 1) < 0.05), (emp, exp)


def test_fft_expectation_approaches_continuous_theory():
    """With a large periodic screen the expected D(r) approaches the closed form at
    lags of a few pixels (the missing power is below 1/(S dx) and above Nyquist)."""
    S, dx, r0, L0 = 1024, 0.02, 0.1, 25.0
    lags = np.array([4, 8, 16])
    exp = at.structure_function_expected_fft(S, dx, r0, L0, lags)
    th = at.structure_function_von_karman(lags * dx, r0, L0)
    assert np.all(np.abs(exp / th - 1) < 0.06), (exp, th)


def test_kolmogorov_screen_structure_function_6p88():
    """Kolmogorov variant (L0 = inf): Monte-Carlo D(r) of the screens agrees with
    the FFT-method expectation, and that expectation climbs towards
    6.88 (r/r0)^5/3 as the screen grows (the deficit is the power below 1/(S dx),
    which an FFT screen without subharmonics cannot hold)."""
    S, dx, r0 = 256, 0.02, 0.1
    lags = np.array([2, 4, 8])
    acc = np.zeros(lags.size)
    n = 24
    for seed in range(n):
        acc += _empirical_D(at.phase_screen_rad(S, dx, r0, math.inf, screen_white_noise(S, 900 + seed)), lags)
    emp = acc / n
    assert np.all(np.abs(emp / at.structure_function_expected_fft(S, dx, r0, math.inf, lags) - 1) < 0.06)
    ratios = [at.structure_function_expected_fft(s, dx, r0, math.inf, lags)
              / at.structure_function_kolmogorov(lags * dx, r0) for s in (256, 1024, 4096)]
    assert np.all(ratios[0] < ratios[1]) and np.all(ratios[1] < ratios[2]) and np.all(ratios[2] < 1.0)
    assert np.all(ratios[2] > 0.85)


def test_bilinear_integer_shift_is_exact_copy_and_wraps():
    g = np.random.default_rng(2)
    scr = g.standard_normal((32, 32))
    i = np.arange(8, dtype=float)
    I, J = np.meshgrid(i, i, indexing="ij")
    out = at.bilinear_sample(scr, I - 3.0, J + 5.0)
    assert np.array_equal(out, scr[np.ix_((np.arange(8) - 3) % 32, (np.arange(8) + 5) % 32)])
    # a shift by the screen size is the identity
    assert np.array_equal(at.bilinear_sample(scr, I + 32.0, J - 64.0), scr[:8, :8])


def test_bilinear_reproduces_linear_function_and_midpoints():
    S = 64
    x = np.arange(S, dtype=float)
    plane = 0.7 * x[:, None] - 1.3 * x[None, :] + 2.0
    I, J = np.meshgrid(np.arange(10, 20, dtype=float), np.arange(10, 20, dtype=float), indexing="ij")
    out = at.bilinear_sample(plane, I + 0.37, J - 0.81)
    assert np.max(np.abs(out - (0.7 * (I + 0.37) - 1.3 * (J - 0.81) + 2.0))) < 1e-12
    scr = np.random.default_rng(4).standard_normal((S, S))
    mid = at.bilinear_sample(scr, I + 0.5, J)
    assert np.max(np.abs(mid - 0.5 * (scr[10:20, 10:20] + scr[11:21, 10:20]))) < 1e-12


def test_atmo_opd_sums_layers_and_moves_with_wind():
    cfg = tiny_config(S=64)
    scr = np.random.default_rng(1).standard_normal((2, 64, 64))
    vel = ((1.0, 0.0), (0.0, 2.0))
    o0 = at.atmo_opd(scr, vel, 0, 16)
    assert np.allclose(o0, scr[0, :16, :16] + scr[1, :16, :16])
    o3 = at.atmo_opd(scr, vel, 3, 16)
    # layer 0 moved +3 rows: pupil pixel (i, j) now sees screen row i - 3
    expect = scr[0][np.ix_((np.arange(16) - 3) % 64, np.arange(16))] + \
        scr[1][np.ix_(np.arange(16), (np.arange(16) - 6) % 64)]
    assert np.allclose(o3, expect)
    assert cfg.S == 64


def test_layer_r0_scaling():
    """Layer screens scale as f_l^(1/2) in OPD (r0_l = r0 f_l^-3/5)."""
    cfg = tiny_config(S=64)
    w = [screen_white_noise(64, 3)]
    from synth.configs import with_, LayerSpec
    one = at.layer_screens_nm(with_(cfg, layers=(LayerSpec(1.0, 0, 1.0),)), w)
    quarter = at.layer_screens_nm(with_(cfg, layers=(LayerSpec(0.25, 0, 1.0),)), w)
    assert np.allclose(quarter, 0.5 * one)


def test_off_axis_footprint_offsets():
    """An off-axis source moves each layer's footprint by h theta: an integer offset
    is an exact copy of the shifted screen, an offset o equals the wind displacement
    of a step t with t v = -o, and zero offsets leave the on-axis sum unchanged."""
    import math
    rng = np.random.default_rng(4)
    S, Np = 64, 16
    scr = rng.standard_normal((2, S, S))
    vel = [(0.3, -0.2), (0.0, 0.7)]
    on = at.atmo_opd(scr, vel, 5, Np)
    assert np.array_equal(on, at.atmo_opd(scr, vel, 5, Np, [(0.0, 0.0), (0.0, 0.0)]))
    # integer offsets at step 0: a plain window of each screen
    o = at.atmo_opd(scr, [(0.0, 0.0), (0.0, 0.0)], 0, Np, [(3.0, -2.0), (-5.0, 4.0)])
    ref = sum(np.roll(np.roll(scr[l], -int(dx), 0), -int(dy), 1)[:Np, :Np]
              for l, (dx, dy) in enumerate([(3, -2), (-5, 4)]))
    assert np.max(np.abs(o - ref)) < 1e-12
    # offset = -t v reproduces step t of the on-axis sum (to float64 rounding)
    t = 7
    off = [(-t * vx, -t * vy) for vx, vy in vel]
    assert np.max(np.abs(at.atmo_opd(scr, vel, 0, Np, off) - at.atmo_opd(scr, vel, t, Np))) < 1e-9
    # geometry: 10 arcsec at 45 degrees, layers at 0 and 8 km, 3.5 cm pixels
    oo = at.footprint_offsets_px([0.0, 8000.0], 10.0, 45.0, 0.035)
    theta = 10.0 / 206264.80624709636                    # arcseconds per radian
    assert oo[0] == (0.0, 0.0)
    assert abs(oo[1][0] - 8000.0 * theta * math.cos(math.pi / 4) / 0.035) < 1e-9
    assert abs(oo[1][0] - oo[1][1]) < 1e-9 and oo[1][0] > 0


def test_cone_effect_scales_a_tilt_layer():
    """Bilinear interpolation reproduces a linear screen exactly, so a tilt layer at
    height h seen from a source at height H shows its slope times 1 - h/H (the cone
    effect reduces the tilt a laser guide star sees), centred on the pupil centre;
    a scale of one leaves the sum unchanged."""
    S, Np = 128, 20
    x = np.arange(S, dtype=np.float64)
    a, b = 0.75, -1.25                        # nm per pixel along axes 0 and 1
    tilt = a * x[:, None] + b * x[None, :]
    scr = np.stack([tilt, np.zeros((S, S))])
    vel = [(0.0, 0.0), (0.0, 0.0)]
    H, h = 90000.0, 12000.0
    sc = at.footprint_scales([h, 0.0], H)
    assert sc[0] == 1.0 - h / H and sc[1] == 1.0
    off = [(30.0, 40.0), (0.0, 0.0)]
    o = at.atmo_opd(scr, vel, 0, Np, off, sc)
    i = np.arange(Np, dtype=np.float64)
    c = (Np - 1) / 2.0
    want = a * (c + 30.0 + (i[:, None] - c) * sc[0]) + b * (c + 40.0 + (i[None, :] - c) * sc[0])
    assert np.max(np.abs(o - want)) < 1e-9
    gx = np.diff(o, axis=0).mean()
    assert abs(gx / a - (1.0 - h / H)) < 1e-12
    rng = np.random.default_rng(2)
    scr2 = rng.standard_normal((2, S, S))
    assert np.array_equal(at.atmo_opd(scr2, [(0.4, 0.1), (0.0, -0.3)], 9, Np, None, [1.0, 1.0]),
                          at.atmo_opd(scr2, [(0.4, 0.1), (0.0, -0.3)], 9, Np))
