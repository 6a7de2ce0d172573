"""GPU atmosphere, DM, reconstructor and detector noise against the oracle."""
import math

import numpy as np
import pytest

from synth import get_config, tiny_config
from synth.configs import with_
from synth.inputs import random_matrix, random_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1607_07624_gb300 import pas
    ctx = pas.pas_ctx_create()
    yield torch, pas, ctx
    torch.cuda.synchronize()
    pas.pas_ctx_destroy(ctx)


def test_atmosphere_matches_oracle_and_integer_shift_is_exact(env):
    torch, pas, ctx = env
    from oracle import atmosphere as at
    S, Np = 256, 60
    scr = np.random.default_rng(3).standard_normal((3, S, S)).astype(np.float32) * 100
    vel = np.array([[0.37, -0.81], [1.0, 0.0], [-2.0, 3.0]])
    d_scr = torch.as_tensor(scr).cuda()
    atmo = pas.pas_atmo_create(ctx, 3, S, Np, vel[:, 0], vel[:, 1], d_scr)
    out = torch.zeros(Np, Np, device="cuda")
    try:
        for step in (0, 1, 7, 123, 1000):
            pas.pas_atmo_advance(atmo, ctx, step, out)
            torch.cuda.synchronize()
            g = out.cpu().numpy().astype(np.float64)
            o = at.atmo_opd(scr.astype(np.float64), vel, step, Np)
            assert np.max(np.abs(g - o)) <= 1e-6 * np.max(np.abs(o)), step
        # integer velocities only: exact copy of the screen sum
        atmo2 = pas.pas_atmo_create(ctx, 2, S, Np, vel[1:, 0], vel[1:, 1], d_scr[1:])
        pas.pas_atmo_advance(atmo2, ctx, 77, out)
        torch.cuda.synchronize()
        o = at.atmo_opd(scr[1:].astype(np.float64), vel[1:], 77, Np).astype(np.float32)
        assert np.array_equal(out.cpu().numpy(), o)
        pas.pas_atmo_destroy(atmo2)
    finally:
        pas.pas_atmo_destroy(atmo)


def test_atmosphere_view_of_an_off_axis_source(env):
    """pas_atmo_create_view: the same screens through footprints moved by per-layer
    offsets (non-integer, as an off-axis source gives), against the oracle."""
    torch, pas, ctx = env
    from oracle import atmosphere as at
    S, Np = 256, 60
    scr = np.random.default_rng(8).standard_normal((3, S, S)).astype(np.float32) * 100
    vel = np.array([[0.37, -0.81], [1.0, 0.0], [-2.0, 3.0]])
    off = np.array([[0.0, 0.0], [3.7, -12.25], [-30.5, 41.125]])
    d_scr = torch.as_tensor(scr).cuda()
    base = pas.pas_atmo_create(ctx, 3, S, Np, vel[:, 0], vel[:, 1], d_scr)
    view = pas.pas_atmo_create_view(base, ctx, off[:, 0], off[:, 1])
    out = torch.zeros(Np, Np, device="cuda")
    try:
        for step in (0, 5, 600):
            pas.pas_atmo_advance(view, ctx, step, out)
            torch.cuda.synchronize()
            o = at.atmo_opd(scr.astype(np.float64), vel, step, Np, [tuple(x) for x in off])
            assert np.max(np.abs(out.cpu().numpy() - o)) <= 1e-6 * np.max(np.abs(o)), step
        with pytest.raises(pas.PasError):
            pas.pas_atmo_create_view(base, ctx, np.array([0.0, np.nan, 0.0]), off[:, 1])
    finally:
        pas.pas_atmo_destroy(view)
        pas.pas_atmo_destroy(base)


@pytest.mark.parametrize("Np", [60, 61])
def test_atmosphere_cone_view_of_a_source_at_finite_height(env, Np):
    """pas_atmo_create_cone_view: footprints shrunk by 1 - h/H about the pupil centre
    (odd and even Np put the centre on and between pixels) and moved by offsets,
    against the oracle; scales outside (0, 1] are rejected."""
    torch, pas, ctx = env
    from oracle import atmosphere as at
    S = 256
    scr = np.random.default_rng(9).standard_normal((3, S, S)).astype(np.float32) * 100
    vel = np.array([[0.37, -0.81], [1.0, 0.0], [-2.0, 3.0]])
    off = np.array([[0.0, 0.0], [3.7, -12.25], [-30.5, 41.125]])
    sc = at.footprint_scales([0.0, 4000.0, 16000.0], 90000.0)
    d_scr = torch.as_tensor(scr).cuda()
    base = pas.pas_atmo_create(ctx, 3, S, Np, vel[:, 0], vel[:, 1], d_scr)
    view = pas.pas_atmo_create_cone_view(base, ctx, off[:, 0], off[:, 1], sc)
    out = torch.zeros(Np, Np, device="cuda")
    try:
        for step in (0, 7, 1500):
            pas.pas_atmo_advance(view, ctx, step, out)
            torch.cuda.synchronize()
            o = at.atmo_opd(scr.astype(np.float64), vel, step, Np, [tuple(x) for x in off], sc)
            assert np.max(np.abs(out.cpu().numpy() - o)) <= 1e-6 * np.max(np.abs(o)), step
        for bad in ([1.0, 0.0, 0.5], [1.0, 1.5, 0.5], [1.0, np.nan, 0.5]):
            with pytest.raises(pas.PasError):
                pas.pas_atmo_create_cone_view(base, ctx, off[:, 0], off[:, 1], np.array(bad))
    finally:
        pas.pas_atmo_destroy(view)
        pas.pas_atmo_destroy(base)


@pytest.mark.parametrize("Np,n_modes", [(16, 10), (64, 100), (240, 400)])
def test_dm_shape_and_residual_match_oracle(env, Np, n_modes):
    torch, pas, ctx = env
    from oracle import modal as md
    from oracle import optics as op
    M = md.modal_basis(Np, 0.1, n_modes)
    mask = op.pupil_mask(Np, 0.1)
    dm = pas.pas_dm_create(ctx, M, Np, 0.1)
    try:
        c = random_vector(n_modes, 11, 20.0).astype(np.float32)
        d_c = torch.as_tensor(c).cuda()
        opd = torch.zeros(Np, Np, device="cuda")
        pas.pas_dm_update(dm, ctx, None, None, d_c, opd)
        atm = (np.random.default_rng(2).standard_normal((Np, Np)) * 50).astype(np.float32)
        res = torch.as_tensor(atm).cuda()
        pas.pas_dm_residual(dm, ctx, res, d_c, res)     # in place
        torch.cuda.synchronize()
        ref = md.basis_to_grid(M.astype(np.float32).astype(np.float64), c.astype(np.float64), mask)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(opd.cpu().numpy() - ref)) <= 2e-6 * scale * math.sqrt(n_modes)
        r_ref = np.where(mask, atm.astype(np.float64) - ref, 0.0)
        assert np.max(np.abs(res.cpu().numpy() - r_ref)) <= 2e-6 * (scale + 200) * math.sqrt(n_modes)
        # integrator: cmd += g * dmodes
        dmodes = torch.as_tensor(random_vector(n_modes, 12).astype(np.float32)).cuda()
        gain = torch.full((n_modes,), 0.5, device="cuda")
        c2 = d_c.clone()
        pas.pas_dm_update(dm, ctx, dmodes, gain, c2, None)
        torch.cuda.synchronize()
        assert torch.allclose(c2, d_c + 0.5 * dmodes, rtol=0, atol=1e-6)
    finally:
        pas.pas_dm_destroy(dm)


@pytest.mark.parametrize("Np,n_modes", [(16, 10), (240, 400)])
def test_bf16_dm_basis_within_rounding_of_oracle(env, Np, n_modes):
    """A PAS_BF16 DM: shape and residual equal the oracle's with the basis rounded to
    bfloat16 (float32 sums), and stay within the rounding's statistical error of the
    exact float64 shape."""
    torch, pas, ctx = env
    from oracle import modal as md
    from oracle import optics as op
    M = md.modal_basis(Np, 0.1, n_modes)
    mask = op.pupil_mask(Np, 0.1)
    dm = pas.pas_dm_create(ctx, M, Np, 0.1, pas.PAS_BF16)
    try:
        c = random_vector(n_modes, 31, 20.0).astype(np.float32)
        d_c = torch.as_tensor(c).cuda()
        opd = torch.zeros(Np, Np, device="cuda")
        pas.pas_dm_update(dm, ctx, None, None, d_c, opd)
        atm = (np.random.default_rng(3).standard_normal((Np, Np)) * 50).astype(np.float32)
        res = torch.as_tensor(atm).cuda()
        pas.pas_dm_residual(dm, ctx, res, d_c, res)
        coeffs = torch.zeros(n_modes, device="cuda")
        pas.pas_dm_project(dm, ctx, opd, coeffs)
        torch.cuda.synchronize()
        Mb = torch.as_tensor(M.astype(np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)
        ref_b = md.basis_to_grid(Mb, c.astype(np.float64), mask)
        ref = md.basis_to_grid(M, c.astype(np.float64), mask)
        scale = np.max(np.abs(ref_b))
        got = opd.cpu().numpy()
        assert np.max(np.abs(got - ref_b)) <= 2e-6 * scale * math.sqrt(n_modes)
        r = ref[mask]
        err = got[mask] - r
        # bf16 rounding: relative 2^-9 per element, independent across modes
        assert np.sqrt(np.mean(err ** 2)) <= 2.0 * 2.0 ** -9 * np.sqrt(np.mean(r ** 2))
        r_ref = np.where(mask, atm.astype(np.float64) - ref_b, 0.0)
        assert np.max(np.abs(res.cpu().numpy() - r_ref)) <= 2e-6 * (scale + 200) * math.sqrt(n_modes)
        # projection with the rounded basis
        pref = Mb.T @ got.astype(np.float64)[mask] / mask.sum()
        assert np.max(np.abs(coeffs.cpu().numpy() - pref)) <= 1e-4 * np.max(np.abs(pref))
    finally:
        pas.pas_dm_destroy(dm)


@pytest.mark.parametrize("n_m,n_s", [(100, 416), (400, 1424), (37, 13), (4000, 14312),
                                     # long slope vectors (bulk-copy rows): ragged rows and
                                     # row counts, a last slot shorter than the others
                                     (1001, 5001), (3, 4100), (257, 8192),
                                     # beyond the register-held slopes of the row pipeline:
                                     # the per-warp bulk-copy rings
                                     (50, 20000)])
def test_reconstructor_fp32_and_bf16(env, n_m, n_s):
    torch, pas, ctx = env
    R = random_matrix(n_m, n_s, 21, 1.0 / math.sqrt(n_s)).astype(np.float32)
    s = random_vector(n_s, 22, 0.05).astype(np.float32)
    exact = R.astype(np.float64) @ s.astype(np.float64)
    d_s = torch.as_tensor(s).cuda()
    out = torch.zeros(n_m, device="cuda")
    for prec in (pas.PAS_FP32, pas.PAS_BF16):
        rec = pas.pas_recon_create(ctx, R, prec)
        try:
            pas.pas_recon_apply(rec, ctx, d_s, out)
            torch.cuda.synchronize()
            assert pas.pas_recon_check(rec, ctx) == 0
            g = out.cpu().numpy().astype(np.float64)
            if prec == pas.PAS_FP32:
                tol = 1e-5 * np.max(np.abs(exact)) + 1e-7
                assert np.max(np.abs(g - exact)) <= tol
            else:
                rel = np.sqrt(np.mean((g - exact) ** 2)) / np.sqrt(np.mean(exact ** 2))
                assert rel <= 0.01, rel
        finally:
            pas.pas_recon_destroy(rec)


def test_detector_noise_draws_match_the_kernel_model(env):
    torch, pas, ctx = env
    import kernel_noise_model as nz  # the kernel's float32 draws (not the oracle)
    fr = (np.random.default_rng(7).random((60, 60)) * 3.0).astype(np.float32)
    fr[:5] = 0.0
    photons, npup, ron, seed = 5.3e4, 2848, 0.5, 1000
    d_in = torch.as_tensor(fr).cuda()
    d_out = torch.zeros_like(d_in)
    for frame_index in (0, 17):
        pas.pas_ccd_noise(ctx, d_in, d_out, photons, npup, ron, seed, frame_index)
        torch.cuda.synchronize()
        g = d_out.cpu().numpy().astype(np.float64)
        o = nz.apply_noise(fr.astype(np.float64), photons, npup, ron, seed, frame_index)
        # same float32 decisions on both sides: counts agree; the Gaussian part
        # differs only by the cosine implementations (a few float32 ulps)
        close = np.abs(g - o) <= 1e-5 * np.maximum(1.0, np.abs(o))
        assert close.mean() >= 0.999, close.mean()
    pas.pas_ccd_noise(ctx, d_in, d_out, photons, npup, 0.0, seed, 3)
    torch.cuda.synchronize()
    o = nz.apply_noise(fr.astype(np.float64), photons, npup, 0.0, seed, 3)
    assert np.mean(d_out.cpu().numpy() == o) >= 0.999


def _loop_views(loop, ctx, n_modes, hist):
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import DevView
    bufs = pas.pas_loop_buffers(loop, ctx)
    return DevView.tensor(bufs["wfe"], (hist,), "<f8"), DevView.tensor(bufs["cmd"], (n_modes,))


@pytest.mark.parametrize("source,n_layers", [(None, 2), ((3.0, 40.0), 2), (None, 16)])
def test_tma_tap_staging_equals_the_4byte_copies(source, n_layers):
    """The residual's TMA tap staging (a box of the two screen rows per pupil-row segment,
    taps past the screen's edge from global memory) against the 4-byte copies, on one
    atmosphere and on screens that start 4 bytes into a buffer (which cannot take TMA
    boxes): with winds that carry the footprint around the 128-pixel screens in both
    axes, every step's residual WFE and the command are bit-identical, on axis and off
    axis."""
    import torch
    from paper_1607_07624_gb300 import pas, calib
    from paper_1607_07624_gb300.system import SCAOSystem
    from synth.configs import LayerSpec
    if n_layers == 2:
        layers = (LayerSpec(0.7, 0.0, 530.0, 30.0), LayerSpec(0.3, 4000.0, 410.0, 200.0))
    else:   # the most layers an atmosphere takes: 16 x 4 segments of boxes per tile
        layers = tuple(LayerSpec(1.0 / n_layers, 500.0 * l, 150.0 + 27.0 * l, 23.0 * l) for l in range(n_layers))
    cfg = with_(tiny_config(Np=64, N=128, n_sub=8, K=8, n_modes=30, S=128), layers=layers)
    s = SCAOSystem(cfg, autotune=False, wfe_history=64, source=source, build_loop=False)
    n = s.d_screens.numel()
    buf = torch.zeros(n + 4, device="cuda", dtype=torch.float32)
    buf[1:1 + n].copy_(s.d_screens.reshape(-1))
    vel = calib.wind_shift_px(cfg)
    atmo_m = pas.pas_atmo_create(s.ctx, len(cfg.layers), cfg.S, cfg.Np, vel[:, 0], vel[:, 1], buf[1:1 + n])
    view_m = None
    if source is not None:
        off = np.array(calib.footprint_offsets_px([ly.height_m for ly in cfg.layers], source[0], source[1], cfg.dx),
                       dtype=np.float64).reshape(-1, 2)
        view_m = pas.pas_atmo_create_view(atmo_m, s.ctx, off[:, 0], off[:, 1])
    pyrs, loops = [], []
    try:
        assert pas.pas_atmo_tma(s.atmo) == 1 and pas.pas_atmo_tma(view_m or atmo_m) == 0
        with pytest.raises(pas.PasError):
            pas.pas_atmo_set_tap_staging(view_m or atmo_m, s.ctx, pas.PAS_TAPS_TMA)
        for atmo, mode in ((s.atmo, pas.PAS_TAPS_TMA), (s.atmo, pas.PAS_TAPS_COPY), (view_m or atmo_m, None)):
            if mode is not None:
                pas.pas_atmo_set_tap_staging(atmo, s.ctx, mode)
            # a sensor per loop (its intermediates), all of one geometry and reference
            pyr = pas.pas_pyr_create(s.ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm,
                                     cfg.obs, s.valid)
            pas.pas_pyr_set_reference(pyr, s.ctx, s.d_sn)
            pyrs.append(pyr)
            loops.append(pas.pas_loop_create(s.ctx, atmo, pyr, s.rec, s.dm, s.d_gain, s.delay, 64))
        n_steps = 60   # about 4 px per step: the footprints wrap around the screen twice
        for loop in loops:
            pas.pas_loop_step(loop, s.ctx, n_steps)
        torch.cuda.synchronize()
        views = [_loop_views(loop, s.ctx, s.n_modes, 64) for loop in loops]
        w0, c0 = views[0][0].cpu().numpy(), views[0][1].cpu().numpy()
        assert np.all(np.isfinite(w0)) and w0[:n_steps].min() > 0.0
        for w, c in views[1:]:
            assert np.array_equal(w.cpu().numpy(), w0)
            assert np.array_equal(c.cpu().numpy(), c0)
        assert pas.pas_atmo_check(s.atmo_base)[0] == pas.PAS_OK
    finally:
        for loop in loops:
            pas.pas_loop_destroy(loop)
        for pyr in pyrs:
            pas.pas_pyr_destroy(pyr)
        if view_m is not None:
            pas.pas_atmo_destroy(view_m)
        pas.pas_atmo_destroy(atmo_m)
        s.close()


def test_tma_tap_staging_wait_gives_up_and_is_reported():
    """A staging wait limit of 0 gives up at once: the residual kernel flags the
    atmosphere, waits for its copies with the long bound and computes the same values;
    pas_atmo_check reports PAS_ETIMEOUT once, and the context stays usable."""
    import torch
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    cfg = tiny_config(Np=64, N=128, n_sub=8, K=8, n_modes=30, S=128)
    ref = SCAOSystem(cfg, autotune=False, wfe_history=64, build_loop=False)
    s = SCAOSystem(cfg, autotune=False, wfe_history=64, build_loop=False, R=ref.R, basis=ref.basis)
    loop = None
    try:
        pas.pas_atmo_set_tap_staging(ref.atmo, ref.ctx, pas.PAS_TAPS_TMA)
        ref_loop = pas.pas_loop_create(ref.ctx, ref.atmo, ref.pyr, ref.rec, ref.dm, ref.d_gain, ref.delay, 64)
        ref.loop = ref_loop
        ref.loop_cmd = _loop_views(ref_loop, ref.ctx, ref.n_modes, 64)[1]
        pas.pas_atmo_set_tap_staging(s.atmo, s.ctx, pas.PAS_TAPS_TMA)
        pas.pas_atmo_set_wait_limit(s.atmo, s.ctx, 0)
        loop = pas.pas_loop_create(s.ctx, s.atmo, s.pyr, s.rec, s.dm, s.d_gain, ref.delay, 64)
        pas.pas_loop_step(ref_loop, ref.ctx, 10)
        pas.pas_loop_step(loop, s.ctx, 10)
        torch.cuda.synchronize()
        st, fault = pas.pas_atmo_check(s.atmo)
        assert st == pas.PAS_ETIMEOUT and fault == 1
        assert pas.pas_atmo_check(s.atmo) == (pas.PAS_OK, 0)
        from paper_1607_07624_gb300.system import DevView
        cmd = DevView.tensor(pas.pas_loop_buffers(loop, s.ctx)["cmd"], (ref.n_modes,)).cpu().numpy()
        assert np.array_equal(ref.loop_cmd.cpu().numpy(), cmd)
        assert pas.pas_atmo_check(ref.atmo)[0] == pas.PAS_OK
    finally:
        if loop is not None:
            pas.pas_loop_destroy(loop)
        s.close()
        ref.close()
