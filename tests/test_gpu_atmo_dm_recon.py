"""GPU atmosphere, DM, reconstructor and detector noise against the oracle."""
import math

import numpy as np
import pytest

from synth import get_config, tiny_config
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
