"""GPU Shack-Hartmann sensor (pas_sh_*) against the FP64 oracle, element by element.

Tolerances (FP32 path): frame max |dI| <= 1e-5 max I_oracle; slopes max |ds| <=
1e-5 max |s_oracle| + 2e-5 pixel. The valid lenslet map is compared bit for bit.
"""
import math

import numpy as np
import pytest

from synth.inputs import random_opd_nm, screen_white_noise

pytestmark = pytest.mark.gpu

LAM = 750.0


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1607_07624_gb300 import pas
    assert torch.cuda.is_available()
    ctx = pas.pas_ctx_create()
    yield torch, pas, ctx
    torch.cuda.synchronize()
    pas.pas_ctx_destroy(ctx)


def open_loop_opd(Np, dx, seed):
    from oracle import atmosphere as at
    S = max(64, 1 << (2 * Np - 1).bit_length())
    scr = at.phase_screen_rad(S, dx, 0.15, 25.0, screen_white_noise(S, seed))
    return (scr[:Np, :Np] * 500.0 / (2 * math.pi)).astype(np.float32)


def run_sh(env, Np, n_sub, ovs, obs, opd32, ref=None):
    torch, pas, ctx = env
    h = pas.pas_sh_create(ctx, Np, n_sub, ovs, LAM, obs)
    try:
        side = pas.pas_sh_frame_side(h)
        nv = pas.pas_sh_n_valid(h)
        fr = torch.zeros(side, side, device="cuda")
        sl = torch.zeros(2 * nv, device="cuda")
        if ref is not None:
            pas.pas_sh_set_reference(h, ctx, torch.as_tensor(ref).cuda())
        pas.pas_sh_measure(h, ctx, torch.as_tensor(opd32).cuda(), fr, sl)
        torch.cuda.synchronize()
        return fr.cpu().numpy().astype(np.float64), sl.cpu().numpy().astype(np.float64), pas.pas_sh_get_valid(h, ctx)
    finally:
        pas.pas_sh_destroy(h)


@pytest.mark.parametrize("Np,n_sub,ovs,obs,kind", [
    (64, 16, 2, 0.1, "small"), (64, 8, 2, 0.1, "open"), (48, 16, 2, 0.1, "open"), (120, 10, 2, 0.0, "small"),
    (64, 4, 2, 0.1, "small"), (240, 30, 2, 0.1, "small"), (240, 30, 2, 0.1, "open"), (96, 12, 3, 0.2, "open")])
def test_sh_matches_oracle(env, Np, n_sub, ovs, obs, kind):
    from oracle import optics as op
    from oracle import shack_hartmann as sh
    opd = random_opd_nm(Np, 60.0, seed=Np + n_sub).astype(np.float32) if kind == "small" \
        else open_loop_opd(Np, 8.4 / Np, Np + 7 * n_sub)
    fr, sl, valid = run_sh(env, Np, n_sub, ovs, obs, opd)
    assert np.array_equal(valid, op.valid_subapertures(Np, obs, n_sub))
    fo, so = sh.sh_measure(opd.astype(np.float64), LAM, obs, n_sub, ovs)
    assert np.max(np.abs(fr - fo)) <= 1e-5 * fo.max()
    assert np.max(np.abs(sl - so)) <= 1e-5 * np.max(np.abs(so)) + 2e-5


def test_reference_cancels_and_tilt_sign(env):
    torch, pas, ctx = env
    Np, n_sub, ovs = 64, 8, 2
    flat = np.zeros((Np, Np), np.float32)
    _, ref, _ = run_sh(env, Np, n_sub, ovs, 0.1, flat)
    _, s0, _ = run_sh(env, Np, n_sub, ovs, 0.1, flat, ref=ref.astype(np.float32))
    assert np.max(np.abs(s0)) == 0.0
    # a small tilt along axis 0 moves every x centroid the same positive way
    b = Np // n_sub
    tilt = np.repeat((0.05 * LAM * np.arange(Np) / b)[:, None], Np, 1).astype(np.float32)
    _, st, _ = run_sh(env, Np, n_sub, ovs, 0.1, tilt, ref=ref.astype(np.float32))
    nv = st.size // 2
    assert np.all(st[:nv] > 0.05) and np.max(np.abs(st[nv:])) < 1e-4


def test_bad_arguments_are_rejected(env):
    torch, pas, ctx = env
    with pytest.raises(pas.PasError):
        pas.pas_sh_create(ctx, 64, 10, 2, LAM, 0.1)     # 10 does not divide 64
    with pytest.raises(pas.PasError):
        pas.pas_sh_create(ctx, 60, 20, 1, LAM, 0.1)     # spot side 3 is odd
    with pytest.raises(pas.PasError):
        pas.pas_sh_create(ctx, 64, 2, 2, LAM, 0.1)      # spot side 64 > 32
    with pytest.raises(pas.PasError):
        pas.pas_sh_create(ctx, 64, 8, 2, LAM, 0.1, valid=np.array([3, 2], np.int32))


def test_sh_closed_loop_matches_oracle(env):
    """The loop with the Shack-Hartmann sensor (pas_loop_create_sh through
    SCAOSystem(sensor="sh")) against the oracle's closed loop with the oracle sensor:
    calibration, then per-step residual WFE."""
    from oracle import atmosphere as at
    from oracle import control as ct
    from oracle import modal as md
    from oracle import optics as op
    from oracle import shack_hartmann as shm
    from paper_1607_07624_gb300.system import SCAOSystem
    from synth import get_config
    from synth.inputs import layer_seeds
    cfg = get_config("scao_8m_64px")
    ovs = 2
    noises = [screen_white_noise(cfg.S, s) for s in layer_seeds(cfg.seed, len(cfg.layers))]
    screens = at.layer_screens_nm(cfg, noises)
    M = md.modal_basis(cfg.Np, cfg.obs, cfg.n_modes)
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    mask = op.pupil_mask(cfg.Np, cfg.obs)
    meas = lambda o, ref=None: shm.sh_measure(o, cfg.wavelength_nm, cfg.obs, cfg.n_sub, ovs, valid, ref)
    sn = meas(np.zeros((cfg.Np, cfg.Np)))[1]
    IM = md.interaction_matrix(lambda o: meas(o, sn)[1], M, mask, cfg.pushpull_nm)
    R = md.pseudo_inverse(IM)
    n = 100
    wo = ct.closed_loop(cfg, screens, M, R, sn, valid, n, sensor=lambda o, t: meas(o, sn))["wfe"]
    s = SCAOSystem(cfg, screens=screens.astype(np.float32), basis=M, R=R, wfe_history=n, sensor="sh", sh_ovs=ovs)
    try:
        assert np.max(np.abs(s.d_sn.cpu().numpy() - sn)) <= 1e-5 * np.max(np.abs(sn)) + 2e-5
        s.calibrate_reconstructor()
        assert np.max(np.abs(s.IM - IM)) <= 1e-3 * np.max(np.abs(IM))
        step, last = s.step(n, stats=True)
        assert step == n
        wg = s.wfe_nm(n)
        assert abs(last - wg[-1]) == 0.0
        assert np.max(np.abs(wg - wo)) <= 2.0, np.max(np.abs(wg - wo))
        assert wg[10:].min() < 0.5 * wg[0]
    finally:
        s.close()


def test_sh_detector_noise_matches_kernel_model_counts(env):
    """Photon and read noise on the Shack-Hartmann frame against the kernel model's
    draws (the float32 decisions of the detector kernel, not the oracle) on the same
    noiseless float32 frame; the slopes are the noisy frame's centroids. The noise
    law itself is judged against the oracle in test_gpu_noise_statistics."""
    torch, pas, ctx = env
    import kernel_noise_model as nz  # the kernel's float32 draws (not the oracle)
    from oracle import shack_hartmann as shm
    Np, n_sub, ovs, obs = 64, 8, 2, 0.1
    opd = random_opd_nm(Np, 60.0, seed=5).astype(np.float32)
    n_pupil = int(pas.pas_pupil_pixels(Np, obs).size)
    photons, ron, seed = 30.0 * n_pupil, 0.5, 77
    h = pas.pas_sh_create(ctx, Np, n_sub, ovs, LAM, obs)
    try:
        side, nv = pas.pas_sh_frame_side(h), pas.pas_sh_n_valid(h)
        fr = torch.zeros(side, side, device="cuda")
        sl = torch.zeros(2 * nv, device="cuda")
        d_opd = torch.as_tensor(opd).cuda()
        pas.pas_sh_measure(h, ctx, d_opd, fr)
        torch.cuda.synchronize()
        clean = fr.cpu().numpy().astype(np.float64)
        for fi, r in ((3, ron), (4, 0.0)):
            pas.pas_sh_set_noise(h, ctx, photons, r, seed, fi)
            pas.pas_sh_measure(h, ctx, d_opd, fr, sl)
            torch.cuda.synchronize()
            g = fr.cpu().numpy().astype(np.float64)
            o = nz.apply_noise(clean, photons, n_pupil, r, seed, fi)
            if r > 0:
                close = np.abs(g - o) <= 1e-5 * np.maximum(1.0, np.abs(o))
                assert close.mean() >= 0.999, close.mean()
            else:
                assert np.mean(g == o) >= 0.999
            so = shm.sh_slopes(g, pas.pas_sh_get_valid(h, ctx), n_sub)
            assert np.max(np.abs(sl.cpu().numpy() - so)) <= 1e-5 * np.max(np.abs(so)) + 2e-5
        # the counter advanced by one per noisy measurement
        pas.pas_sh_measure(h, ctx, d_opd, fr)
        torch.cuda.synchronize()
        assert np.mean(fr.cpu().numpy() == nz.apply_noise(clean, photons, n_pupil, 0.0, seed, 5)) >= 0.999
    finally:
        pas.pas_sh_destroy(h)


@pytest.mark.parametrize("n_int,noisy", [(3, False), (2, True)])
def test_sh_integrating_detector_loop_matches_oracle(env, n_int, noisy):
    """The Shack-Hartmann loop with a detector integrating n_int steps per frame
    (pas_loop_set_integration) against the oracle loop integrating the oracle sensor's
    frames (mean frame at (t + 1) mod n_int = 0, noise on it, command held between).
    With noise, the oracle loop is fed the kernel model's draws (same counts)."""
    from oracle import atmosphere as at
    from oracle import control as ct
    from oracle import modal as md
    import kernel_noise_model as nz  # the kernel's float32 draws (not the oracle)
    from oracle import optics as op
    from oracle import shack_hartmann as shm
    from paper_1607_07624_gb300 import pas as P
    from paper_1607_07624_gb300.system import SCAOSystem
    from synth import get_config
    from synth.inputs import layer_seeds
    cfg = get_config("scao_8m_64px")
    ovs = 2
    noises = [screen_white_noise(cfg.S, s) for s in layer_seeds(cfg.seed, len(cfg.layers))]
    screens = at.layer_screens_nm(cfg, noises)
    M = md.modal_basis(cfg.Np, cfg.obs, cfg.n_modes)
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    mask = op.pupil_mask(cfg.Np, cfg.obs)
    meas = lambda o, ref=None: shm.sh_measure(o, cfg.wavelength_nm, cfg.obs, cfg.n_sub, ovs, valid, ref)
    sn = meas(np.zeros((cfg.Np, cfg.Np)))[1]
    R = md.pseudo_inverse(md.interaction_matrix(lambda o: meas(o, sn)[1], M, mask, cfg.pushpull_nm))
    noise, kw = None, {}
    if noisy:
        n_pupil = int(P.pas_pupil_pixels(cfg.Np, cfg.obs).size)
        photons, ron, seed = 2.0e5, 0.5, 17
        noise = lambda fr, t: nz.apply_noise(fr, photons, n_pupil, ron, seed, t)
        kw["noise"] = (photons, ron, seed)
    n = 36
    ref = ct.closed_loop(cfg, screens, M, R, sn, valid, n, noise=noise, n_int=n_int, record=True,
                         sensor=lambda o, t: meas(o), slopes_of=lambda f: shm.sh_slopes(f, valid, cfg.n_sub, sn))
    s = SCAOSystem(cfg, screens=screens.astype(np.float32), basis=M, R=R, wfe_history=n, sensor="sh", sh_ovs=ovs,
                   detector_steps=n_int, **kw)
    try:
        cmds = []
        for t in range(n):
            s.step(1)
            cmds.append(s.loop_cmd.cpu().numpy().copy())
        wg = s.wfe_nm(n)
        assert np.max(np.abs(wg - ref["wfe"])) <= 2.0, np.max(np.abs(wg - ref["wfe"]))
        cmds = np.array(cmds)
        for t in range(1, n):
            if (t + 1) % n_int != 0:
                assert np.array_equal(cmds[t], cmds[t - 1]), t
        assert np.max(np.abs(cmds - ref["cmd"])) <= 1e-2 * np.max(np.abs(ref["cmd"])), \
            np.max(np.abs(cmds - ref["cmd"]))
    finally:
        s.close()
