"""Pins of the oracle's optics against the mathematics (no GPU).

Each test fixes a fact that does not come from the oracle's own code: a brute-force
sum, a closed-form transform, an invariant (unitarity, Parseval, symmetry), or a
physical sign fixed by the stated DFT / mask / tilt conventions.
"""
import math

import numpy as np
import pytest

from oracle import optics as op
from synth import get_config, tiny_config
from synth.inputs import random_opd_nm


def brute_force_cdft2(E):
    N = E.shape[0]
    c = (N - 1) / 2.0
    out = np.zeros((N, N), dtype=complex)
    for u in range(N):
        for v in range(N):
            acc = 0j
            for x in range(N):
                for y in range(N):
                    ph = -2 * math.pi * ((x - c) * (u - c) + (y - c) * (v - c)) / N
                    acc += E[x, y] * complex(math.cos(ph), math.sin(ph))
            out[u, v] = acc / N
    return out


@pytest.mark.parametrize("N", [8, 12, 15, 16])
def test_cdft2_matches_brute_force(N):
    g = np.random.default_rng(N)
    E = g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))
    assert np.max(np.abs(op.cdft2(E) - brute_force_cdft2(E))) < 1e-12
    assert np.max(np.abs(op.cdft2_fft(E) - brute_force_cdft2(E))) < 1e-12


@pytest.mark.parametrize("N", [8, 15, 32, 48])
def test_unitary_and_inverse(N):
    W = op.centred_dft_matrix(N)
    assert np.allclose(W @ np.conj(W).T, np.eye(N), atol=1e-12)
    g = np.random.default_rng(1)
    E = g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))
    assert np.max(np.abs(op.icdft2(op.cdft2(E)) - E)) < 1e-12
    assert np.max(np.abs(op.icdft2_fft(op.cdft2_fft(E)) - E)) < 1e-12


def test_gaussian_is_self_dual_and_shift_theorem_sign():
    """exp(-pi x~^2/N) maps to exp(-pi u~^2/N) (continuous FT, aliasing ~e^-pi N/4);
    a shift by +a multiplies the transform by exp(-2 pi i a u~ / N)."""
    N = 64
    t = np.arange(N) - (N - 1) / 2.0
    g1 = np.exp(-math.pi * t ** 2 / N)
    X = op.cdft2(np.outer(g1, np.ones(N)) * 0 + np.outer(g1, g1))
    assert np.max(np.abs(X - np.outer(g1, g1))) < 1e-12
    a = 3
    gs = np.exp(-math.pi * (t - a) ** 2 / N)
    Xs = op.cdft2(np.outer(gs, g1))
    expect = np.outer(g1 * np.exp(-2j * math.pi * a * t / N), g1)
    assert np.max(np.abs(Xs - expect)) < 1e-10


def test_real_centrosymmetric_input_has_real_transform():
    N = 16
    g = np.random.default_rng(3).standard_normal((N, N))
    E = g + g[::-1, ::-1]
    assert np.max(np.abs(op.cdft2(E).imag)) < 1e-12


def test_pupil_mask_counts_and_area():
    for Np, obs in [(64, 0.1), (240, 0.1), (480, 0.1), (16, 0.0)]:
        m = op.pupil_mask(Np, obs)
        # brute force with float geometry: centre distance vs radius
        cnt = 0
        r_out = Np / 2.0
        r_in = obs * Np / 2.0
        for i in range(Np):
            for j in range(Np):
                d = math.hypot(i - (Np - 1) / 2.0, j - (Np - 1) / 2.0)
                if d <= r_out + 1e-12 and d >= r_in - 1e-12:
                    cnt += 1
        assert m.sum() == cnt
        area = math.pi / 4 * Np * Np * (1 - obs * obs)
        assert abs(m.sum() - area) / area < 1.0 / Np
    assert op.pupil_mask(64, 0.1).sum() == 3196
    assert op.pupil_mask(240, 0.1).sum() == 44796


def test_pyramid_mask_structure():
    N = 32
    P = op.pyramid_mask(N, N / 4)
    assert np.allclose(np.abs(P), 1.0)
    # separable: P(u, v) = p(u) p(v)
    p = P[:, N // 2] / np.sqrt(P[N // 2, N // 2])
    assert np.allclose(P, np.outer(p, p))
    # each face is a linear phase: for u~ > 0 consecutive ratio exp(i 2 pi delta / N)
    r = P[N // 2 + 1:, 0] / P[N // 2:-1, 0]
    assert np.allclose(r, np.exp(2j * math.pi * (N / 4) / N))


@pytest.mark.parametrize("cfgkind", ["tiny", "cfg1"])
def test_parseval_through_pyramid_and_binning(cfgkind):
    cfg = tiny_config() if cfgkind == "tiny" else get_config("scao_8m_64px")
    opd = random_opd_nm(cfg.Np, 300.0, seed=11)
    frame, _ = op.pwfs_measure(opd, cfg)
    npix = op.pupil_mask(cfg.Np, cfg.obs).sum()
    assert abs(frame.sum() - npix) / npix < 1e-12


def test_flat_wavefront_symmetries():
    cfg = get_config("scao_8m_64px")
    n = cfg.n_sub
    frame, s = op.pwfs_measure(np.zeros((cfg.Np, cfg.Np)), cfg)
    q00, q01, q10, q11 = frame[:n, :n], frame[:n, n:], frame[n:, :n], frame[n:, n:]
    tot = [q.sum() for q in (q00, q01, q10, q11)]
    assert np.ptp(tot) / np.mean(tot) < 1e-12
    # the four images are mirror images of one another
    assert np.max(np.abs(q01 - q00[:, ::-1])) < 1e-12
    assert np.max(np.abs(q10 - q00[::-1, :])) < 1e-12
    assert np.max(np.abs(q11 - q00[::-1, ::-1])) < 1e-12
    nv = s.size // 2
    assert abs(s[:nv].mean()) < 1e-14 and abs(s[nv:].mean()) < 1e-14
    # per-sub-aperture flat slopes are not zero (edge diffraction); after the
    # reference they are zero exactly
    assert np.max(np.abs(s)) > 0.05
    valid = op.valid_subapertures(cfg.Np, cfg.obs, n)
    assert np.max(np.abs(op.pwfs_slopes(frame, valid, n, sn=s))) == 0.0


def test_tilt_sign_orthogonality_and_linearity():
    """A tilt +a (lambda/D) along axis 0 moves the focal spot to u~ > 0; that face's
    phase exp(+i 2 pi delta u~ / N) shifts its image by -delta, so the low-row
    images brighten and Sx < 0. Sy stays zero by symmetry; the response is odd
    and linear for small a."""
    cfg = get_config("scao_8m_64px")
    X, Y = op.pixel_coords(cfg.Np)
    _, s0 = op.pwfs_measure(np.zeros((cfg.Np, cfg.Np)), cfg)
    nv = s0.size // 2
    resp = {}
    for a in (0.01, 0.02, 0.05, -0.05, 1.0):
        _, s = op.pwfs_measure(a * cfg.wavelength_nm * X, cfg, sn=s0)
        resp[a] = (s[:nv].mean(), s[nv:].mean())
    assert resp[0.05][0] < 0
    assert abs(resp[0.05][1]) < 1e-12
    assert abs(resp[0.05][0] + resp[-0.05][0]) < 1e-12
    g = [resp[a][0] / a for a in (0.01, 0.02, 0.05)]
    assert np.ptp(g) / abs(np.mean(g)) < 0.005
    # optical gain: at a = R/3 the response per lambda/D has clearly dropped
    assert 0.4 < resp[1.0][0] / g[0] < 0.8
    # y tilt gives Sy only
    _, s = op.pwfs_measure(0.05 * cfg.wavelength_nm * Y, cfg, sn=s0)
    assert s[nv:].mean() < 0 and abs(s[:nv].mean()) < 1e-12


def test_modulation_gain_falls_with_radius():
    base = tiny_config(Np=32, N=64, n_sub=8, K=24)
    X, _ = op.pixel_coords(base.Np)
    gains = []
    for R in (3.0, 6.0, 10.0):
        from synth.configs import with_
        cfg = with_(base, mod_radius=R, K=max(24, int(8 * R)))
        _, s0 = op.pwfs_measure(np.zeros((cfg.Np, cfg.Np)), cfg)
        _, s = op.pwfs_measure(0.02 * cfg.wavelength_nm * X, cfg, sn=s0)
        gains.append(-s[: s.size // 2].mean() / 0.02)
    assert gains[0] > gains[1] > gains[2] > 0
    # roughly inverse to the radius
    assert 0.3 < gains[1] / gains[0] * 2 < 1.5


def test_modulation_converges_with_K():
    from synth.configs import with_
    base = tiny_config(Np=16, N=32, n_sub=4, mod_radius=3.0)
    opd = random_opd_nm(16, 200.0, seed=5)
    frames = {K: op.pwfs_measure(opd, with_(base, K=K))[0] for K in (8, 16, 32, 128)}
    d = [np.abs(frames[K] - frames[128]).max() for K in (8, 16, 32)]
    assert d[0] > d[1] > d[2]


def test_binning_and_slopes_brute_force():
    g = np.random.default_rng(9)
    I = g.random((24, 24))
    b = 3
    fr = op.bin_detector(I, b)
    for p in range(8):
        for q in range(8):
            assert abs(fr[p, q] - sum(I[p * b + i, q * b + j] for i in range(b) for j in range(b))) < 1e-12
    n = 4
    frame = g.random((2 * n, 2 * n)) + 0.5
    valid = np.array([1, 2, 5, 6, 9, 10, 13, 14], dtype=np.int32)
    s = op.pwfs_slopes(frame, valid, n)
    tots = []
    for v in valid:
        r, c = divmod(int(v), n)
        tots.append(frame[r, c] + frame[r, n + c] + frame[n + r, c] + frame[n + r, n + c])
    F = sum(tots) / len(tots)
    for k, v in enumerate(valid):
        r, c = divmod(int(v), n)
        sx = (frame[n + r, c] + frame[n + r, n + c] - frame[r, c] - frame[r, n + c]) / F
        sy = (frame[r, n + c] + frame[n + r, n + c] - frame[r, c] - frame[n + r, c]) / F
        assert abs(s[k] - sx) < 1e-12 and abs(s[len(valid) + k] - sy) < 1e-12


def test_valid_subapertures_rule_and_counts():
    for Np, ns, expect in [(64, 16, 208), (240, 30, 712), (480, 96, 7156)]:
        v = op.valid_subapertures(Np, 0.1, ns)
        assert v.size == expect
        assert np.all(np.diff(v) > 0)
    # brute force on a small case
    Np, ns = 32, 8
    m = op.pupil_mask(Np, 0.1)
    b = Np // ns
    ref = [r * ns + c for r in range(ns) for c in range(ns)
           if 2 * int(m[r * b:(r + 1) * b, c * b:(c + 1) * b].sum()) >= b * b]
    assert list(op.valid_subapertures(Np, 0.1, ns)) == ref


def test_threshold_acquisition_agrees_with_geometric_rule():
    """Table 3's procedure: a flat frame at 20 lambda/D modulation, thresholded,
    finds (nearly) the geometric valid set."""
    from synth.configs import with_
    cfg = with_(get_config("scao_8m_64px"), mod_radius=20.0, K=160)
    frame, _ = op.pwfs_measure(np.zeros((cfg.Np, cfg.Np)), cfg)
    geo = set(op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub).tolist())
    thr = set(op.valid_subapertures_threshold(frame, cfg.n_sub, 0.5).tolist())
    assert len(geo ^ thr) <= 0.1 * len(geo)


# ---------------------------------------------------------------- fractional binning

def test_rebin_is_block_sum_for_integer_binning():
    I = np.random.default_rng(41).random((48, 48))
    assert np.max(np.abs(op.rebin(I, 12) - op.bin_detector(I, 4))) < 1e-12
    assert np.max(np.abs(op.detector_frame(I, 6) - op.bin_detector(I, 4))) == 0.0


@pytest.mark.parametrize("N,nd", [(128, 20), (96, 18), (50, 7), (64, 10)])
def test_rebin_equals_upsampled_block_sum_and_keeps_the_total(N, nd):
    """Brute force: split every fine pixel into nd x nd equal micro-pixels; a detector
    pixel is then exactly N x N micro-pixels."""
    I = np.random.default_rng(N + nd).random((N, N))
    up = np.kron(I, np.ones((nd, nd))) / (nd * nd)
    brute = up.reshape(nd, N, nd, N).sum(axis=(1, 3))
    fr = op.rebin(I, nd)
    assert np.max(np.abs(fr - brute)) < 1e-10 * I.sum()
    assert abs(fr.sum() - I.sum()) < 1e-10 * I.sum()
    O = op.overlap_units(N, nd)
    assert np.all(O.sum(axis=0) == nd)          # each fine pixel is fully shared out
    assert np.all(O.sum(axis=1) == N)           # each detector pixel covers b fine pixels


@pytest.mark.parametrize("Np,n_sub", [(64, 16), (96, 12), (128, 20), (96, 18), (50, 7)])
def test_valid_rule_by_micro_pixel_counts(Np, n_sub):
    mask = op.pupil_mask(Np, 0.1)
    up = np.kron(mask.astype(np.int64), np.ones((n_sub, n_sub), dtype=np.int64))
    A_bf = up.reshape(n_sub, Np, n_sub, Np).sum(axis=(1, 3))
    assert np.array_equal(op.subaperture_area_units(mask, n_sub), A_bf)
    v = op.valid_subapertures(Np, 0.1, n_sub)
    assert np.array_equal(v, np.flatnonzero((2 * A_bf).ravel() >= Np * Np))
    if Np % n_sub == 0:
        b = Np // n_sub
        assert np.array_equal(v, np.flatnonzero((2 * op.subaperture_counts(mask, n_sub)).ravel() >= b * b))
