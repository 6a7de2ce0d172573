"""Pins of the oracle Shack-Hartmann sensor (oracle/shack_hartmann.py) against what
the mathematics fixes: a brute-force DFT per lenslet, Parseval per spot, the point
symmetry of flat spots, the exact roll of whole-wave tilts, the reflection given by
the conjugate field and the sign and size of the centroid response to small tilts."""
import math

import numpy as np
import pytest

from oracle import optics as op
from oracle import shack_hartmann as sh

LAM = 750.0


def _opd(Np, rms, seed):
    return np.random.default_rng(seed).standard_normal((Np, Np)) * rms


@pytest.mark.parametrize("Np,n_sub,ovs,obs", [(4, 2, 2, 0.0), (6, 2, 2, 0.1), (8, 4, 3, 0.0)])
def test_frame_equals_brute_force_dft(Np, n_sub, ovs, obs):
    opd = _opd(Np, 300.0, Np + ovs)
    A = op.pupil_mask(Np, obs)
    b = Np // n_sub
    M = ovs * b
    ref = np.zeros((n_sub * M, n_sub * M))
    for r in range(n_sub):
        for c in range(n_sub):
            for k in range(M):
                for l in range(M):
                    s = 0j
                    for i in range(b):
                        for j in range(b):
                            ii, jj = r * b + i, c * b + j
                            if A[ii, jj]:
                                s += np.exp(2j * math.pi * opd[ii, jj] / LAM) * \
                                    np.exp(-2j * math.pi * ((k - M // 2) * i + (l - M // 2) * j) / M)
                    ref[r * M + k, c * M + l] = abs(s) ** 2 / M ** 2
    assert np.max(np.abs(sh.sh_frame(opd, LAM, obs, n_sub, ovs) - ref)) < 1e-12


def test_parseval_per_spot():
    Np, n_sub, ovs = 40, 5, 2
    A = op.pupil_mask(Np, 0.1)
    fr = sh.sh_frame(_opd(Np, 500.0, 2), LAM, 0.1, n_sub, ovs)
    b, M = Np // n_sub, 2 * Np // n_sub
    for r in range(n_sub):
        for c in range(n_sub):
            lit = A[r * b:(r + 1) * b, c * b:(c + 1) * b].sum()
            assert abs(fr[r * M:(r + 1) * M, c * M:(c + 1) * M].sum() - lit) < 1e-9 * max(lit, 1)


def test_flat_spots_are_point_symmetric_and_reference_cancels():
    Np, n_sub, ovs = 32, 4, 2
    M = 2 * Np // n_sub
    fr = sh.sh_frame(np.zeros((Np, Np)), LAM, 0.0, n_sub, ovs)
    idx = (M - np.arange(M)) % M
    for r in (1, 2):
        for c in (1, 2):                      # fully lit lenslets: real symmetric field
            I = fr[r * M:(r + 1) * M, c * M:(c + 1) * M]
            assert np.max(np.abs(I - I[idx][:, idx])) < 1e-12
    valid = op.valid_subapertures(Np, 0.0, n_sub)
    ref = sh.sh_slopes(fr, valid, n_sub)
    assert np.max(np.abs(sh.sh_slopes(fr, valid, n_sub, ref))) == 0.0


@pytest.mark.parametrize("m,axis", [(1, 0), (-1, 1), (2, 0)])
def test_whole_wave_tilt_rolls_every_spot_by_m_ovs(m, axis):
    Np, n_sub, ovs = 24, 3, 2
    b, M = Np // n_sub, ovs * Np // n_sub
    ramp = m * LAM * np.arange(Np, dtype=np.float64) / b
    opd = np.repeat(ramp[:, None], Np, 1) if axis == 0 else np.repeat(ramp[None, :], Np, 0)
    f0 = sh.sh_frame(np.zeros((Np, Np)), LAM, 0.1, n_sub, ovs)
    f1 = sh.sh_frame(opd, LAM, 0.1, n_sub, ovs)
    for r in range(n_sub):
        for c in range(n_sub):
            s0 = f0[r * M:(r + 1) * M, c * M:(c + 1) * M]
            s1 = f1[r * M:(r + 1) * M, c * M:(c + 1) * M]
            assert np.max(np.abs(s1 - np.roll(s0, m * ovs, axis=axis))) < 1e-11


def test_conjugate_field_reflects_every_spot():
    Np, n_sub, ovs = 16, 2, 2
    M = ovs * Np // n_sub
    opd = _opd(Np, 200.0, 4)
    idx = (M - np.arange(M)) % M
    fa = sh.sh_frame(opd, LAM, 0.1, n_sub, ovs)
    fb = sh.sh_frame(-opd, LAM, 0.1, n_sub, ovs)
    for r in range(n_sub):
        for c in range(n_sub):
            a = fa[r * M:(r + 1) * M, c * M:(c + 1) * M]
            bb = fb[r * M:(r + 1) * M, c * M:(c + 1) * M]
            assert np.max(np.abs(bb - a[idx][:, idx])) < 1e-12


@pytest.mark.parametrize("t", [0.01, 0.05])
def test_small_tilt_moves_the_centroid_by_about_ovs_t(t):
    """A tilt of t waves across each lenslet along axis 0 moves the spot by ovs t
    pixels; the centre of gravity over the M-pixel window sees 0.93 of it (the
    window truncates the sinc^2 wings) and nothing on the other axis."""
    Np, n_sub, ovs = 32, 4, 2
    b = Np // n_sub
    opd = np.repeat((t * LAM * np.arange(Np, dtype=np.float64) / b)[:, None], Np, 1)
    cx0, cy0 = sh.centroids(sh.sh_frame(np.zeros((Np, Np)), LAM, 0.0, n_sub, ovs), n_sub)
    cx, cy = sh.centroids(sh.sh_frame(opd, LAM, 0.0, n_sub, ovs), n_sub)
    gain = (cx - cx0)[1:3, 1:3] / (ovs * t)
    assert np.all((gain > 0.85) & (gain < 1.0))
    assert np.max(np.abs((cy - cy0)[1:3, 1:3])) < 1e-12


def test_integrating_detector_of_a_frozen_atmosphere_subsamples_the_single_rate_loop():
    """The Shack-Hartmann loop with a detector integrating 3 steps: with no wind and
    delay 1 every frame of a window is the same, so window k repeats step k of the
    single-rate loop (WFE, command changing only at the read-out, and the read-out
    frame equal to the single frame: the mean, not the sum)."""
    from oracle import atmosphere as at
    from oracle import control as ct
    from oracle import modal as md
    from synth import tiny_config
    from synth.configs import LayerSpec
    from synth.inputs import screen_white_noise
    cfg = tiny_config(Np=16, N=32, n_sub=4, K=8, n_modes=12, mod_radius=2.0, S=64, r0_m=0.5,
                      layers=(LayerSpec(1.0, 0.0, 0.0),))
    mask = op.pupil_mask(cfg.Np, cfg.obs)
    M = md.modal_basis(cfg.Np, cfg.obs, cfg.n_modes)
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    meas = lambda o, ref=None: sh.sh_measure(o, LAM, cfg.obs, cfg.n_sub, 2, valid, ref)
    sn = meas(np.zeros((cfg.Np, cfg.Np)))[1]
    R = md.pseudo_inverse(md.interaction_matrix(lambda o: meas(o, sn)[1], M, mask, 5.0))
    screens = at.layer_screens_nm(cfg, [screen_white_noise(cfg.S, 21)])
    n = 3
    one = ct.closed_loop(cfg, screens, M, R, sn, valid, 4, delay=1, record=True, sensor=lambda o, t: meas(o, sn))
    mr = ct.closed_loop(cfg, screens, M, R, sn, valid, 4 * n, delay=1, record=True, n_int=n,
                        sensor=lambda o, t: meas(o, sn), slopes_of=lambda f: sh.sh_slopes(f, valid, cfg.n_sub, sn))
    for k in range(4):
        for i in range(n):
            assert abs(mr["wfe"][n * k + i] - one["wfe"][k]) <= 1e-9 * one["wfe"][k]
            want = one["cmd"][k] if i == n - 1 else (one["cmd"][k - 1] if k > 0 else np.zeros(cfg.n_modes))
            assert np.max(np.abs(mr["cmd"][n * k + i] - want)) <= 1e-9 * np.max(np.abs(one["cmd"][k]))
        assert np.max(np.abs(mr["frame"][n * k + n - 1] - one["frame"][k])) <= 1e-12 * one["frame"][k].max()
    assert one["wfe"][1] < 0.9 * one["wfe"][0]
