"""GPU PSF camera (pas_psf_*) against the FP64 oracle, element by element.

Tolerances (FP32 path): PSF max |dP| <= 1e-5 * max P_oracle; Strehl |dSR| <= 1e-5.
The oracle promotes the same float32 OPD to float64.
"""
import math

import numpy as np
import pytest

from synth import get_config
from synth.inputs import random_opd_nm, screen_white_noise

pytestmark = pytest.mark.gpu

LAM = 1650.0


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


def gpu_psf(env, Np, nd, obs, opd32, accumulate_with=None):
    torch, pas, ctx = env
    h = pas.pas_psf_create(ctx, Np, nd, LAM, obs)
    try:
        N = pas.pas_psf_size(h)
        assert N == nd * Np
        d_opd = torch.as_tensor(opd32).cuda()
        out = torch.zeros(N, N, device="cuda")
        sr = torch.zeros(1, dtype=torch.float64, device="cuda")
        pas.pas_psf_compute(h, ctx, d_opd, out, False, sr)
        if accumulate_with is not None:
            pas.pas_psf_compute(h, ctx, torch.as_tensor(accumulate_with).cuda(), out, True, None)
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64), float(sr.item())
    finally:
        pas.pas_psf_destroy(h)


@pytest.mark.parametrize("Np,nd,obs,kind", [(64, 2, 0.1, "small"), (64, 4, 0.1, "open"), (64, 8, 0.0, "small"),
                                            (48, 8, 0.25, "open"), (64, 3, 0.1, "open"), (120, 4, 0.1, "small"), (240, 4, 0.1, "open"),
                                            (240, 8, 0.1, "small"), (240, 8, 0.1, "open"), (240, 3, 0.1, "open"),
                                            (240, 5, 0.0, "small"), (240, 16, 0.1, "small"), (480, 2, 0.1, "open"),
                                            (480, 4, 0.1, "small"), (480, 3, 0.2, "open")])
def test_psf_matches_oracle(env, Np, nd, obs, kind):
    from oracle import psf as ps
    if kind == "small":
        opd = random_opd_nm(Np, 80.0, seed=Np + nd).astype(np.float32)   # closed-loop-like residual
    else:
        opd = open_loop_opd(Np, 8.4 / Np, Np * nd)                          # open loop, several waves
    P, sr = gpu_psf(env, Np, nd, obs, opd)
    Po = ps.psf(opd.astype(np.float64), LAM, obs, nd)
    assert np.max(np.abs(P - Po)) <= 1e-5 * Po.max()
    assert abs(sr - ps.strehl(opd.astype(np.float64), LAM, obs)) <= 1e-5
    assert abs(sr - P[nd * Np // 2, nd * Np // 2]) <= 1e-7


def test_flat_wavefront_peaks_at_one_in_the_centre(env):
    Np, nd = 240, 8
    P, sr = gpu_psf(env, Np, nd, 0.1, np.zeros((Np, Np), np.float32))
    N = nd * Np
    assert abs(sr - 1.0) < 1e-6 and int(np.argmax(P)) == (N // 2) * N + N // 2
    n_pup = env[1].pas_pupil_pixels(Np, 0.1).size
    assert abs(P.sum() - N * N / n_pup) <= 1e-5 * N * N / n_pup        # Parseval


def test_integrated_psf_accumulates(env):
    from oracle import psf as ps
    Np, nd = 64, 4
    a = random_opd_nm(Np, 150.0, seed=5).astype(np.float32)
    b = random_opd_nm(Np, 300.0, seed=6).astype(np.float32)
    P, _ = gpu_psf(env, Np, nd, 0.1, a, accumulate_with=b)
    ref = ps.integrated_psf([a.astype(np.float64), b.astype(np.float64)], LAM, 0.1, nd)
    assert np.max(np.abs(P - ref)) <= 1e-5 * ref.max()


def test_bad_arguments_are_rejected(env):
    torch, pas, ctx = env
    with pytest.raises(pas.PasError):
        pas.pas_psf_create(ctx, 60, 4, LAM, 0.1)      # 60 px is not a supported FFT length
    with pytest.raises(pas.PasError):
        pas.pas_psf_create(ctx, 64, 17, LAM, 0.1)
    with pytest.raises(pas.PasError):
        pas.pas_psf_create(ctx, 64, 0, LAM, 0.1)
    with pytest.raises(pas.PasError):
        pas.pas_psf_create(ctx, 64, 4, -1.0, 0.1)
    h = pas.pas_psf_create(ctx, 64, 4, LAM, 0.1)
    try:
        with pytest.raises(pas.PasError):
            pas.pas_psf_compute(h, ctx, None, torch.zeros(256, 256, device="cuda"))
    finally:
        pas.pas_psf_destroy(h)


@pytest.mark.parametrize("name,nd", [("scao_8m_64px", 4), ("scao_lbt_240px", 3)])
def test_camera_in_the_closed_loop_matches_oracle(env, name, nd):
    """SCAOSystem.attach_camera: from the start step on, each step's PSF of the loop's
    residual is integrated and its Strehl ratio recorded (against the oracle on the
    same float32 residuals, copied after every step). At 240 px the camera runs the
    paired transforms (odd padding: a warp's second residue empty)."""
    torch, pas, ctx = env
    from oracle import psf as ps
    from paper_1607_07624_gb300.system import SCAOSystem
    cfg = get_config(name)
    s = SCAOSystem(cfg, wfe_history=64)
    try:
        N = s.attach_camera(nd=nd, wavelength_nm=LAM, start_step=2)
        assert N == nd * cfg.Np
        opds = []
        for _ in range(6):
            s.step(1)
            torch.cuda.synchronize()
            opds.append(s.loop_opd.cpu().numpy().astype(np.float64))
        ref = ps.integrated_psf(opds, LAM, cfg.obs, nd, start=2)
        P = s.int_psf.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(P - ref)) <= 1e-5 * ref.max()
        sr = s.sr.cpu().numpy()
        for t in range(6):
            want = ps.strehl(opds[t], LAM, cfg.obs) if t >= 2 else 0.0
            assert abs(sr[t] - want) <= 1e-5, (t, sr[t], want)
        s.detach_camera()
        s.step(2)                       # without the camera the loop runs on
    finally:
        s.close()


@pytest.mark.parametrize("name,nd", [("scao_8m_64px", 4), ("scao_lbt_240px", 2)])
def test_camera_inside_the_step_graph_equals_the_camera_called_per_step(env, name, nd):
    """The camera inside the loop's step graph (its passes beside the sensor, the step
    counter read on the device) gives the integrated PSF and the Strehl ring of the camera
    called after every step, bit for bit, and the loop's own WFE is unchanged by it; a
    persistent batch refuses the loop while the camera is attached, and the camera
    detaches cleanly."""
    torch, pas, ctx = env
    from paper_1607_07624_gb300.system import SCAOSystem
    cfg = get_config(name)
    a = SCAOSystem(cfg, wfe_history=64, autotune=False)
    b = SCAOSystem(cfg, wfe_history=64, autotune=False, basis=a.basis, R=a.R)
    try:
        a.attach_camera(nd=nd, wavelength_nm=LAM, start_step=3, in_graph=True)
        b.attach_camera(nd=nd, wavelength_nm=LAM, start_step=3, in_graph=False)
        assert a._cam_in_graph and not b._cam_in_graph
        a.step(12)
        b.step(12)
        torch.cuda.synchronize()
        assert np.array_equal(a.int_psf.cpu().numpy(), b.int_psf.cpu().numpy())
        assert np.array_equal(a.sr.cpu().numpy(), b.sr.cpu().numpy())
        assert np.all(a.sr.cpu().numpy()[:3] == 0.0) and np.all(a.sr.cpu().numpy()[3:12] > 0.0)
        assert np.array_equal(a.wfe_nm(12), b.wfe_nm(12))
        with pytest.raises(pas.PasError, match="camera"):
            pas.pas_batch_create_ex(a.ctx, [a.loop], pas.PAS_BATCH_PERSISTENT)
        a.detach_camera()
        a.step(2)
        b.detach_camera()
        b.step(2)
        torch.cuda.synchronize()
        assert np.array_equal(a.wfe_nm(14), b.wfe_nm(14))
    finally:
        b.close()
        a.close()
