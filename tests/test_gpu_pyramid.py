"""GPU pyramid (pas_pyr_measure) against the FP64 oracle, element by element.

Inputs are seeded OPD maps in float32; the oracle promotes the same float32 values
to float64, so the test judges the pyramid path alone. Tolerances (FP32 path):
  frame:  max |dI| <= 1e-5 * max |I_oracle|
  slopes: max |ds| <= 1e-5 * max |s_oracle| + 1e-7
Index maps (valid sub-apertures) are compared bit for bit.
"""
import math

import numpy as np
import pytest

from synth import get_config, tiny_config
from synth.configs import with_
from synth.inputs import random_opd_nm, screen_white_noise

pytestmark = pytest.mark.gpu

FRAME_TOL = 1e-5
SLOPE_TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1607_07624_gb300 import pas
    assert torch.cuda.is_available()
    ctx = pas.pas_ctx_create()
    yield torch, pas, ctx
    torch.cuda.synchronize()
    pas.pas_ctx_destroy(ctx)


def open_loop_opd(cfg, seed):
    """An open-loop atmospheric OPD sample (tens of radians) from an oracle screen."""
    from oracle import atmosphere as at
    S = max(64, 1 << (2 * cfg.Np - 1).bit_length())
    scr = at.phase_screen_rad(S, cfg.dx, cfg.r0_m, cfg.L0_m, screen_white_noise(S, seed))
    return scr[:cfg.Np, :cfg.Np] * 500.0 / (2 * math.pi)


def run_gpu(env, cfg, opd32, valid=None):
    torch, pas, ctx = env
    pyr = pas.pas_pyr_create(ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm,
                             cfg.obs, valid)
    try:
        d_opd = torch.as_tensor(opd32).cuda()
        nv = pas.pas_pyr_n_valid(pyr)
        fr = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
        sl = torch.zeros(2 * nv, device="cuda")
        pas.pas_pyr_measure(pyr, ctx, d_opd, fr, sl)
        torch.cuda.synchronize()
        return fr.cpu().numpy().astype(np.float64), sl.cpu().numpy().astype(np.float64), \
            pas.pas_pyr_get_valid(pyr, ctx)
    finally:
        pas.pas_pyr_destroy(pyr)


def oracle_measure(cfg, opd32, valid):
    from oracle import optics as op
    I = op.pwfs_intensity(opd32.astype(np.float64), cfg.wavelength_nm, cfg.obs, cfg.N, cfg.K,
                          cfg.mod_radius, cfg.delta)
    fr = op.detector_frame(I, cfg.n_sub)
    return fr, op.pwfs_slopes(fr, valid, cfg.n_sub)


def check(cfg, fr_g, sl_g, fr_o, sl_o):
    ef = np.max(np.abs(fr_g - fr_o)) / np.max(np.abs(fr_o))
    es = np.max(np.abs(sl_g - sl_o))
    assert ef <= FRAME_TOL, f"{cfg.name}: frame rel err {ef:.3e}"
    assert es <= SLOPE_TOL * np.max(np.abs(sl_o)) + 1e-7, f"{cfg.name}: slope err {es:.3e}"
    return ef, es


TINY = [
    tiny_config(Np=8, N=16, n_sub=2, K=4),          # radices 4,4
    tiny_config(Np=12, N=24, n_sub=3, K=6),         # 3,8
    tiny_config(Np=20, N=40, n_sub=5, K=5),         # 5,8, odd K (no shared rows pass)
    tiny_config(Np=24, N=48, n_sub=4, K=8),         # 3,4,4, b = 6
    tiny_config(Np=40, N=80, n_sub=10, K=12),       # 5,4,4
    tiny_config(Np=60, N=120, n_sub=10, K=12, mod_radius=3.0),  # 5,3,8
    tiny_config(Np=16, N=32, n_sub=4, K=1, mod_radius=0.0),     # unmodulated
    tiny_config(Np=80, N=160, n_sub=20, K=16, obs=0.3),
    tiny_config(Np=96, N=192, n_sub=16, K=8),
    tiny_config(Np=120, N=240, n_sub=24, K=10),
    # the four-step engine's lengths: four transforms per warp at N = 256 (K = 7 and 2
    # leave a call partly empty), two at N = 480 (odd K leaves a warp's last pair half
    # empty), one at N = 960
    tiny_config(Np=128, N=256, n_sub=16, K=7, mod_radius=3.0),
    tiny_config(Np=128, N=256, n_sub=32, K=2),
    tiny_config(Np=320, N=640, n_sub=40, K=7, mod_radius=3.0),   # pass-by-pass engine, odd K
    tiny_config(Np=240, N=480, n_sub=30, K=5, mod_radius=3.0),
    tiny_config(Np=480, N=960, n_sub=96, K=3, mod_radius=4.0),
]


@pytest.mark.parametrize("cfg", TINY, ids=lambda c: f"N{c.N}_K{c.K}")
def test_small_grids_match_oracle(env, cfg):
    from oracle import optics as op
    opd = random_opd_nm(cfg.Np, 250.0, seed=cfg.N + cfg.K).astype(np.float32)
    fr_g, sl_g, valid = run_gpu(env, cfg, opd)
    assert np.array_equal(valid, op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub))
    check(cfg, fr_g, sl_g, *oracle_measure(cfg, opd, valid))


FRACTIONAL = [
    tiny_config(Np=32, N=64, n_sub=5, K=8),                      # 6.4 pixels per sub-aperture
    tiny_config(Np=64, N=128, n_sub=20, K=12),                   # 3.2
    tiny_config(Np=24, N=48, n_sub=7, K=5),                      # 3.43, odd K
    tiny_config(Np=128, N=256, n_sub=20, K=12, mod_radius=3.0),  # 6.4: batched 8 m group
    tiny_config(Np=320, N=640, n_sub=60, K=24, mod_radius=3.0),  # 5.33: batched 25 m group
]


@pytest.mark.parametrize("cfg", FRACTIONAL, ids=lambda c: f"N{c.N}_nsub{c.n_sub}")
def test_non_integer_binning_matches_oracle(env, cfg):
    """Detector pixels of N / (2 n_sub) fine pixels, not an integer: area-weighted
    rebinning (the oracle's exact rational weights) and the rational valid rule."""
    from oracle import optics as op
    assert cfg.N % (2 * cfg.n_sub) != 0
    opd = random_opd_nm(cfg.Np, 250.0, seed=cfg.N + cfg.n_sub).astype(np.float32)
    fr_g, sl_g, valid = run_gpu(env, cfg, opd)
    assert np.array_equal(valid, op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub))
    fr_o, sl_o = oracle_measure(cfg, opd, valid)
    check(cfg, fr_g, sl_g, fr_o, sl_o)
    # the frame keeps the total intensity of the grid
    I = op.pwfs_intensity(opd.astype(np.float64), cfg.wavelength_nm, cfg.obs, cfg.N, cfg.K, cfg.mod_radius,
                          cfg.delta)
    assert abs(fr_g.sum() - I.sum()) <= 1e-5 * I.sum()


@pytest.mark.parametrize("name,k", [("scao_8m_64px", 1), ("scao_lbt_240px", 2), ("scao_elt_480px", 3)])
def test_full_size_configs_open_loop_phase(env, name, k):
    """Full-size N = 128 / 480 / 960 grids on an open-loop screen sample (the phasor
    sees tens of radians)."""
    cfg = get_config(name)
    opd = open_loop_opd(cfg, 4000 + k).astype(np.float32)
    assert np.ptp(opd) * 2 * math.pi / cfg.wavelength_nm > 20.0
    fr_g, sl_g, valid = run_gpu(env, cfg, opd)
    check(cfg, fr_g, sl_g, *oracle_measure(cfg, opd, valid))


def test_four_step_columns_pass_with_odd_and_even_groupings(env):
    """N = 480 (two modulation points per warp call): modulation groups of 7, 3, 2 and
    1 points, and two CTAs per detector column, all against the oracle."""
    torch, pas, ctx = env
    cfg = tiny_config(Np=240, N=480, n_sub=30, K=7, mod_radius=3.0)
    opd = random_opd_nm(cfg.Np, 250.0, seed=17).astype(np.float32)
    from oracle import optics as op
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    fr_o, sl_o = oracle_measure(cfg, opd, valid)
    pyr = pas.pas_pyr_create(ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs)
    try:
        nv = pas.pas_pyr_n_valid(pyr)
        d_opd = torch.as_tensor(opd).cuda()
        for t in [(4, 2, 1, 1), (4, 2, 3, 1), (4, 2, 4, 1), (8, 3, 7, 1), (4, 2, 3, 2), (2, 1, 2, 4)]:
            pas.pas_pyr_set_tuning(pyr, ctx, *t)
            fr = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
            sl = torch.zeros(2 * nv, device="cuda")
            pas.pas_pyr_measure(pyr, ctx, d_opd, fr, sl)
            torch.cuda.synchronize()
            check(cfg, fr.cpu().numpy().astype(np.float64), sl.cpu().numpy().astype(np.float64), fr_o, sl_o)
    finally:
        pas.pas_pyr_destroy(pyr)


def test_flat_wavefront_and_parseval(env):
    from oracle import optics as op
    cfg = get_config("scao_8m_64px")
    fr_g, sl_g, valid = run_gpu(env, cfg, np.zeros((cfg.Np, cfg.Np), np.float32))
    n = cfg.n_sub
    tots = [fr_g[:n, :n].sum(), fr_g[:n, n:].sum(), fr_g[n:, :n].sum(), fr_g[n:, n:].sum()]
    assert np.ptp(tots) / np.mean(tots) < 1e-5
    assert abs(fr_g.sum() - op.pupil_mask(cfg.Np, cfg.obs).sum()) / fr_g.sum() < 1e-5
    nv = valid.size
    assert abs(sl_g[:nv].mean()) < 1e-6 and abs(sl_g[nv:].mean()) < 1e-6


def test_reference_subtraction_and_user_valid_list(env):
    torch, pas, ctx = env
    from oracle import optics as op
    cfg = tiny_config(Np=24, N=48, n_sub=4, K=8)
    valid = np.array([1, 2, 5, 6, 9, 10], dtype=np.int32)
    opd = random_opd_nm(cfg.Np, 100.0, seed=3).astype(np.float32)
    pyr = pas.pas_pyr_create(ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm,
                             cfg.obs, valid)
    try:
        sn = torch.linspace(-0.1, 0.1, 2 * valid.size, device="cuda")
        pas.pas_pyr_set_reference(pyr, ctx, sn)
        sl = torch.zeros(2 * valid.size, device="cuda")
        pas.pas_pyr_measure(pyr, ctx, torch.as_tensor(opd).cuda(), None, sl)
        torch.cuda.synchronize()
        _, s_o = oracle_measure(cfg, opd, valid)
        s_o = s_o - sn.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(sl.cpu().numpy() - s_o)) <= SLOPE_TOL * np.max(np.abs(s_o)) + 1e-7
    finally:
        pas.pas_pyr_destroy(pyr)


def test_bad_arguments_are_rejected(env):
    torch, pas, ctx = env
    with pytest.raises(pas.PasError) as e:
        pas.pas_pyr_create(ctx, 64, 100, 12, 16, 3.0, 750.0, 0.1)
    assert e.value.status == pas.PAS_EINVAL
    with pytest.raises(pas.PasError):
        pas.pas_pyr_create(ctx, 64, 128, 12, 16, 3.0, 750.0, 0.1, valid=np.array([5, 3], np.int32))
    with pytest.raises(pas.PasError):
        pas.pas_pyr_create(ctx, 36, 72, 4, 4, 3.0, 750.0, 0.1)  # 72 = 8*9 unsupported


def test_autotune_and_tunings_give_the_same_frame(env):
    """Every launch geometry computes the same frame (up to the float32 order of
    the modulation-group sums); the autotuner returns a valid one."""
    torch, pas, ctx = env
    cfg = get_config("scao_8m_64px")
    opd = torch.as_tensor(random_opd_nm(cfg.Np, 300.0, seed=9).astype(np.float32)).cuda()
    pyr = pas.pas_pyr_create(ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs)
    try:
        nv = pas.pas_pyr_n_valid(pyr)
        frames = []
        for t in [(1, 1, 1), (2, 3, 4), (8, 7, 12), (4, 2, 5), (2, 3, 4, 2), (4, 2, 6, 4), (8, 1, 12, 4),
                  (16, 1, 12), (16, 7, 5, 2)]:
            pas.pas_pyr_set_tuning(pyr, ctx, *t)
            fr = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
            sl = torch.zeros(2 * nv, device="cuda")
            pas.pas_pyr_measure(pyr, ctx, opd, fr, sl)
            torch.cuda.synchronize()
            frames.append(fr.cpu().numpy())
        for f in frames[1:]:
            assert np.max(np.abs(f - frames[0])) <= 1e-6 * np.max(frames[0])
        best = pas.pas_pyr_autotune(pyr, ctx, opd, 2)
        assert best[0] in (2, 4, 8, 16) and 1 <= best[1] and 1 <= best[2] <= cfg.K
        b = cfg.N // cfg.n_det
        assert best[3] >= 1 and b % best[3] == 0
        assert pas.pas_pyr_get_tuning(pyr, ctx) == best
        with pytest.raises(pas.PasError):
            pas.pas_pyr_set_tuning(pyr, ctx, 3, 1, 1)
        with pytest.raises(pas.PasError):
            pas.pas_pyr_set_tuning(pyr, ctx, 4, 1, 1, 3)    # 3 does not divide b = 4
    finally:
        pas.pas_pyr_destroy(pyr)


@pytest.mark.parametrize("name,rows", [("scao_lbt_240px", [(2, 1), (4, 7), (8, 13), (16, 3), (16, 13)]),
                                       ("scao_elt_480px", [(2, 17), (4, 5), (8, 5), (16, 3), (16, 6)])])
def test_rows_pass_geometry_leaves_the_frame_bit_identical(env, name, rows):
    """The rows pass's geometry (pupil rows per CTA, 16 included, and sin values per
    CTA) changes which warp transforms which row, not the arithmetic: with the columns
    geometry fixed, frame and slopes are bit-identical (the persistent batched launch
    relies on it)."""
    torch, pas, ctx = env
    cfg = get_config(name)
    opd = torch.as_tensor(random_opd_nm(cfg.Np, 200.0, seed=23).astype(np.float32)).cuda()
    pyr = pas.pas_pyr_create(ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs)
    try:
        nv = pas.pas_pyr_n_valid(pyr)
        out = []
        for r, chunks in rows:
            pas.pas_pyr_set_tuning(pyr, ctx, r, chunks, 5, 1)
            fr = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
            sl = torch.zeros(2 * nv, device="cuda")
            pas.pas_pyr_measure(pyr, ctx, opd, fr, sl)
            torch.cuda.synchronize()
            out.append((fr.cpu().numpy(), sl.cpu().numpy()))
        for fr, sl in out[1:]:
            assert np.array_equal(fr, out[0][0]) and np.array_equal(sl, out[0][1])
    finally:
        pas.pas_pyr_destroy(pyr)


@pytest.mark.parametrize("Np,N,n_sub,rows", [(128, 256, 16, [(2, 1), (4, 7), (8, 3), (16, 2)]),
                                             (320, 640, 40, [(2, 1), (4, 7), (8, 3), (8, 2)])])
def test_launch_geometry_leaves_the_frame_bit_identical(env, Np, N, n_sub, rows):
    """N = 256 (the four-step engine, four transforms per call: sin chunks that leave calls
    partly empty) and N = 640 (the pass-by-pass engine): rows-pass geometries give the same
    frame and slopes bit for bit, and every columns-pass grouping (kper 12, 4, 3, 1)
    matches the oracle."""
    from oracle import optics as op
    torch, pas, ctx = env
    cfg = tiny_config(Np=Np, N=N, n_sub=n_sub, K=12, mod_radius=3.0)
    opd32 = random_opd_nm(cfg.Np, 200.0, seed=29).astype(np.float32)
    opd = torch.as_tensor(opd32).cuda()
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    fr_o, sl_o = oracle_measure(cfg, opd32, valid)
    pyr = pas.pas_pyr_create(ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs)
    try:
        nv = pas.pas_pyr_n_valid(pyr)
        assert nv == valid.size
        out = {}
        for r, chunks, groups in [(r, c, 3) for r, c in rows] + [(4, 2, 1), (4, 2, 4), (4, 2, 12)]:
            pas.pas_pyr_set_tuning(pyr, ctx, r, chunks, groups, 1)
            fr = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
            sl = torch.zeros(2 * nv, device="cuda")
            pas.pas_pyr_measure(pyr, ctx, opd, fr, sl)
            torch.cuda.synchronize()
            out.setdefault(groups, []).append((fr.cpu().numpy(), sl.cpu().numpy()))
        for fr, sl in out[3][1:]:
            assert np.array_equal(fr, out[3][0][0]) and np.array_equal(sl, out[3][0][1])
        for runs in out.values():
            check(cfg, runs[0][0].astype(np.float64), runs[0][1].astype(np.float64), fr_o, sl_o)
    finally:
        pas.pas_pyr_destroy(pyr)


@pytest.mark.parametrize("name,tunings", [("scao_8m_64px", [None, (2, 1, 3, 2), (2, 1, 3, 4)]),
                                          ("scao_lbt_240px", [None])])
def test_noise_inside_the_pyramid_matches_kernel_model_counts(env, name, tunings):
    """Photon and read noise drawn by the columns pass (the last CTA of each detector
    column; lanes of a group share a pixel's rejection loop) against the kernel
    model's draws (the detector kernel's float32 decisions, not the oracle) on the
    same noiseless float32 frame: the grouped draw equals the sequential one. The column splits put 4, 2 and 1 lanes
    on each pixel of the 64 px case."""
    torch, pas, ctx = env
    import kernel_noise_model as nz  # the kernel's float32 draws (not the oracle)
    cfg = get_config(name)
    opd = torch.as_tensor(open_loop_opd(cfg, 21).astype(np.float32)).cuda()
    n_pupil = int(pas.pas_pupil_pixels(cfg.Np, cfg.obs).size)
    photons, ron, seed = 40.0 * n_pupil, 0.5, 1234
    pyr = pas.pas_pyr_create(ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs)
    try:
        fr = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
        for t in tunings:
            if t is not None:
                pas.pas_pyr_set_tuning(pyr, ctx, *t)
            pas.pas_pyr_set_noise(pyr, ctx, 0.0, 0.0, 0, 0)
            pas.pas_pyr_measure(pyr, ctx, opd, fr)
            torch.cuda.synchronize()
            clean = fr.cpu().numpy()
            lam = clean.astype(np.float64) * photons / n_pupil
            assert (lam < 10).any() and (lam >= 10).any()          # both Poisson branches
            for fi, r in ((5, ron), (6, 0.0)):
                pas.pas_pyr_set_noise(pyr, ctx, photons, r, seed, fi)
                pas.pas_pyr_measure(pyr, ctx, opd, fr)
                torch.cuda.synchronize()
                g = fr.cpu().numpy().astype(np.float64)
                o = nz.apply_noise(clean.astype(np.float64), photons, n_pupil, r, seed, fi)
                if r > 0:
                    close = np.abs(g - o) <= 1e-5 * np.maximum(1.0, np.abs(o))
                    assert close.mean() >= 0.999, (t, close.mean())
                else:
                    assert np.mean(g == o) >= 0.999, (t, np.mean(g == o))
    finally:
        pas.pas_pyr_destroy(pyr)


EXTENDED = [
    # (config, ex, ey, w): asymmetric sources, repeated ey values (shared rows passes),
    # odd K, zero and unequal weights
    (tiny_config(Np=24, N=48, n_sub=4, K=8), [0.0, 1.5, -0.75, 1.5], [0.5, 0.5, -1.25, 2.0], [1.0, 2.0, 0.5, 0.0]),
    (tiny_config(Np=20, N=40, n_sub=5, K=5), [0.3], [-0.9], None),
    (tiny_config(Np=32, N=64, n_sub=8, K=12), None, None, None),   # a 3 lambda/D disc, 5 x 5 grid
]


@pytest.mark.parametrize("case", range(len(EXTENDED)))
def test_extended_source_matches_oracle(env, case):
    """pas_pyr_create_extended against the oracle's weighted sum of point sources with
    their wavefront tilts (the kernels ride the points on the modulation circle and
    carry the weights in the column tilts' amplitudes)."""
    torch, pas, ctx = env
    from oracle import optics as op
    from paper_1607_07624_gb300 import calib
    cfg, ex, ey, w = EXTENDED[case]
    if ex is None:
        ex, ey = calib.disc_source(3.0, 5)
    opd = random_opd_nm(cfg.Np, 60.0, seed=40 + case).astype(np.float32)
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    pyr = pas.pas_pyr_create_extended(ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm,
                                      cfg.obs, ex, ey, w)
    try:
        nv = pas.pas_pyr_n_valid(pyr)
        fr = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
        sl = torch.zeros(2 * nv, device="cuda")
        pas.pas_pyr_measure(pyr, ctx, torch.as_tensor(opd).cuda(), fr, sl)
        torch.cuda.synchronize()
        I = op.pwfs_intensity_extended(opd.astype(np.float64), cfg.wavelength_nm, cfg.obs, cfg.N, cfg.K,
                                       cfg.mod_radius, ex, ey, w, cfg.delta)
        fo = op.detector_frame(I, cfg.n_sub)
        check(cfg, fr.cpu().numpy().astype(np.float64), sl.cpu().numpy().astype(np.float64), fo,
              op.pwfs_slopes(fo, valid, cfg.n_sub))
    finally:
        pas.pas_pyr_destroy(pyr)


def test_extended_source_full_size_sampled_and_point_identity(env):
    """The 240 px pyramid (K = 24) with a 3 x 3 grid source of 2 lambda/D: frame
    against the oracle on the same input; a one-point source at the origin is the
    point-source sensor bit for bit; bad sources are rejected."""
    torch, pas, ctx = env
    from oracle import optics as op
    cfg = get_config("scao_lbt_240px")
    g = np.linspace(-1.0, 1.0, 3)
    ex, ey = [a for a in g for _ in g], [b for _ in g for b in g]
    opd = open_loop_opd(cfg, 91).astype(np.float32)
    d_opd = torch.as_tensor(opd).cuda()
    fr = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
    args = (ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs)
    pyr = pas.pas_pyr_create_extended(*args, ex, ey)
    try:
        pas.pas_pyr_measure(pyr, ctx, d_opd, fr)
        torch.cuda.synchronize()
        I = op.pwfs_intensity_extended(opd.astype(np.float64), cfg.wavelength_nm, cfg.obs, cfg.N, cfg.K,
                                       cfg.mod_radius, ex, ey, None, cfg.delta)
        fo = op.detector_frame(I, cfg.n_sub)
        assert np.max(np.abs(fr.cpu().numpy() - fo)) <= FRAME_TOL * fo.max()
    finally:
        pas.pas_pyr_destroy(pyr)
    one = pas.pas_pyr_create_extended(*args, [0.0], [0.0])
    ref = pas.pas_pyr_create(*args)
    f1 = torch.zeros_like(fr)
    try:
        pas.pas_pyr_measure(one, ctx, d_opd, fr)
        pas.pas_pyr_measure(ref, ctx, d_opd, f1)
        torch.cuda.synchronize()
        assert torch.equal(fr, f1)
    finally:
        pas.pas_pyr_destroy(one)
        pas.pas_pyr_destroy(ref)
    for bad in (([0.0, np.nan], [0.0, 0.0], None), ([0.0], [0.0], [-1.0]), ([0.0, 1.0], [0.0, 0.0], [0.0, 0.0])):
        with pytest.raises(pas.PasError):
            pas.pas_pyr_create_extended(*args, *bad)
