"""Pins of the oracle's modal basis, reconstructor, integrator/loop and noise."""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import modal as md
from oracle import control as ct
from oracle import noise as nz
from oracle import optics as op
from oracle import atmosphere as at
from synth import tiny_config
from synth.configs import with_, LayerSpec
from synth.inputs import screen_white_noise


# ---------------------------------------------------------------- Zernike / basis

def test_noll_ordering_matches_published_table():
    for j, n, m in read_golden("noll_indices.txt"):
        assert md.noll_to_nm(int(j)) == (int(n), int(m))


def test_low_order_zernikes_closed_forms():
    g = np.random.default_rng(0)
    rho = g.random(200)
    th = g.uniform(-math.pi, math.pi, 200)
    x, y = rho * np.cos(th), rho * np.sin(th)
    closed = {
        2: 2 * x, 3: 2 * y, 4: math.sqrt(3) * (2 * rho ** 2 - 1),
        5: math.sqrt(6) * 2 * x * y, 6: math.sqrt(6) * (x ** 2 - y ** 2),
        7: math.sqrt(8) * (3 * rho ** 2 - 2) * y, 8: math.sqrt(8) * (3 * rho ** 2 - 2) * x,
        9: math.sqrt(8) * (3 * x ** 2 * y - y ** 3), 10: math.sqrt(8) * (x ** 3 - 3 * x * y ** 2),
        11: math.sqrt(5) * (6 * rho ** 4 - 6 * rho ** 2 + 1),
    }
    for j, z in closed.items():
        assert np.max(np.abs(md.zernike(j, rho, th) - z)) < 1e-12, j


def test_zernikes_unit_rms_on_disc():
    """Noll normalisation: mean of Z_j^2 over the unit disc is 1 (fine polar grid)."""
    nr, nt = 400, 256
    r = (np.arange(nr) + 0.5) / nr
    t = 2 * np.pi * np.arange(nt) / nt
    R, T = np.meshgrid(r, t, indexing="ij")
    w = R / (np.sum(R))
    for j in (2, 4, 7, 11, 16, 22, 37):
        z = md.zernike(j, R, T)
        assert abs(np.sum(w * z * z) - 1) < 2e-3, j
    assert abs(np.sum(w * md.zernike(4, R, T) * md.zernike(11, R, T))) < 1e-3


def test_modal_basis_orthonormal_on_mask():
    M = md.modal_basis(64, 0.1, 100)
    n = M.shape[0]
    assert n == 3196
    assert np.max(np.abs(M.T @ M / n - np.eye(100))) < 1e-10
    # column order kept: mode 0 is tip (linear in x up to the piston removal)
    mask = op.pupil_mask(64, 0.1)
    X, _ = op.pixel_coords(64)
    xx = X[mask]
    corr = np.dot(M[:, 0], xx - xx.mean()) / (np.linalg.norm(M[:, 0]) * np.linalg.norm(xx - xx.mean()))
    assert corr > 0.999999


# ---------------------------------------------------------------- IM / pinv

def test_pinv_identity_and_truncation():
    g = np.random.default_rng(1)
    IM = g.standard_normal((60, 20))
    R = md.pseudo_inverse(IM)
    assert np.max(np.abs(R @ IM - np.eye(20))) < 1e-12
    # a rank-deficient column is dropped: R IM is the projector on the kept space
    IM2 = IM.copy()
    IM2[:, 5] = IM2[:, 4]
    R2 = md.pseudo_inverse(IM2)
    P = R2 @ IM2
    assert np.max(np.abs(P @ P - P)) < 1e-10 and abs(np.trace(P) - 19) < 1e-9


def test_interaction_matrix_mode_in_mode_out():
    cfg = tiny_config(Np=16, N=32, n_sub=4, K=8, n_modes=6, mod_radius=2.0)
    mask = op.pupil_mask(cfg.Np, cfg.obs)
    M = md.modal_basis(cfg.Np, cfg.obs, cfg.n_modes)
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    _, sn = op.pwfs_measure(np.zeros((cfg.Np, cfg.Np)), cfg, valid)
    meas = lambda opd: op.pwfs_measure(opd, cfg, valid, sn)[1]
    IM = md.interaction_matrix(meas, M, mask, amp_nm=5.0)
    R = md.pseudo_inverse(IM)
    for m in range(cfg.n_modes):
        c = np.zeros(cfg.n_modes)
        c[m] = 2.0
        est = R @ meas(md.basis_to_grid(M, c, mask))
        assert np.max(np.abs(est - c)) < 0.02 * 2.0, (m, est)


# ---------------------------------------------------------------- integrator / loop

def test_integrator_closed_form_with_identity_sensor():
    g = 0.5
    a = np.array([3.0, -1.0])
    c = np.zeros(2)
    for t in range(1, 12):
        c = ct.integrator_step(c, a - c, g)
        assert np.allclose(a - c, (1 - g) ** t * a, rtol=0, atol=1e-14)


def test_wfe_removes_piston():
    mask = op.pupil_mask(32, 0.1)
    assert ct.residual_wfe_nm(np.where(mask, 42.0, 0.0), mask) == 0.0
    X, _ = op.pixel_coords(32)
    v = (100 * X)[mask]
    assert abs(ct.residual_wfe_nm(100 * X, mask) - v.std()) < 1e-12


def _tiny_loop_setup(static=True):
    cfg = tiny_config(Np=16, N=32, n_sub=4, K=8, n_modes=12, mod_radius=2.0, S=64,
                      r0_m=0.5, layers=(LayerSpec(1.0, 0.0, 0.0 if static else 2.0),))
    mask = op.pupil_mask(cfg.Np, cfg.obs)
    M = md.modal_basis(cfg.Np, cfg.obs, cfg.n_modes)
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    _, sn = op.pwfs_measure(np.zeros((cfg.Np, cfg.Np)), cfg, valid)
    IM = md.interaction_matrix(lambda o: op.pwfs_measure(o, cfg, valid, sn)[1], M, mask, 5.0)
    R = md.pseudo_inverse(IM)
    return cfg, mask, M, valid, sn, R


def test_zero_atmosphere_stays_exactly_zero():
    cfg, mask, M, valid, sn, R = _tiny_loop_setup()
    screens = np.zeros((1, cfg.S, cfg.S))
    out = ct.closed_loop(cfg, screens, M, R, sn, valid, 6)
    assert np.all(out["wfe"] == 0.0) and np.all(out["cmd"] == 0.0)


def test_static_modal_aberration_decays_geometrically():
    """A static aberration inside the DM space decays as (1-g)^t with delay 1."""
    cfg, mask, M, valid, sn, R = _tiny_loop_setup()
    c_true = np.zeros(cfg.n_modes)
    c_true[[0, 2, 5]] = [3.0, -2.0, 1.5]
    scr = np.zeros((1, cfg.S, cfg.S))
    scr[0, :cfg.Np, :cfg.Np] = md.basis_to_grid(M, c_true, mask)
    out = ct.closed_loop(cfg, scr, M, R, sn, valid, 8, record=True)
    res = np.array([np.linalg.norm(c_true - c) for c in out["cmd"]])
    expect = np.linalg.norm(c_true) * 0.5 ** np.arange(1, 9)
    assert np.all(np.abs(res - expect) < 0.03 * np.linalg.norm(c_true) + 0.05 * expect)


def test_delay_two_lags_one_more_step():
    cfg, mask, M, valid, sn, R = _tiny_loop_setup()
    c_true = np.zeros(cfg.n_modes)
    c_true[1] = 2.0
    scr = np.zeros((1, cfg.S, cfg.S))
    scr[0, :cfg.Np, :cfg.Np] = md.basis_to_grid(M, c_true, mask)
    o1 = ct.closed_loop(cfg, scr, M, R, sn, valid, 3, delay=1)
    o2 = ct.closed_loop(cfg, scr, M, R, sn, valid, 3, delay=2)
    assert o1["wfe"][1] < 0.7 * o1["wfe"][0]
    assert abs(o2["wfe"][1] - o2["wfe"][0]) < 1e-9 and o2["wfe"][2] < 0.7 * o2["wfe"][0]


def test_detector_integration_of_a_frozen_atmosphere_subsamples_the_single_rate_loop():
    """With no wind and delay 1 the command is constant over each detector window, so
    its n_int frames are identical and their mean is the single-step frame: window k
    of the multi-rate loop repeats step k of the single-rate loop (same residual, read
    out at its last step, the command changing only there)."""
    cfg, mask, M, valid, sn, R = _tiny_loop_setup()
    screens = at.layer_screens_nm(cfg, [screen_white_noise(cfg.S, 21)])
    n = 3
    one = ct.closed_loop(cfg, screens, M, R, sn, valid, 4, delay=1, record=True)
    mr = ct.closed_loop(cfg, screens, M, R, sn, valid, 4 * n, delay=1, record=True, n_int=n)
    for k in range(4):
        for i in range(n):
            assert abs(mr["wfe"][n * k + i] - one["wfe"][k]) <= 1e-9 * one["wfe"][k]
            want = one["cmd"][k] if i == n - 1 else (one["cmd"][k - 1] if k > 0 else np.zeros(cfg.n_modes))
            assert np.max(np.abs(mr["cmd"][n * k + i] - want)) <= 1e-9 * np.max(np.abs(one["cmd"][k]))
        # the read-out frame is the window's mean, not its sum (the normalised slopes
        # alone cannot tell them apart)
        assert np.max(np.abs(mr["frame"][n * k + n - 1] - one["frame"][k])) <= 1e-12 * one["frame"][k].max()
    assert one["wfe"][1] < 0.8 * one["wfe"][0]
    base = ct.closed_loop(cfg, screens, M, R, sn, valid, 5)
    assert np.array_equal(ct.closed_loop(cfg, screens, M, R, sn, valid, 5, n_int=1)["wfe"], base["wfe"])


def test_closed_loop_reduces_turbulence_wfe():
    cfg, mask, M, valid, sn, R = _tiny_loop_setup(static=False)
    screens = at.layer_screens_nm(cfg, [screen_white_noise(cfg.S, 77)])
    out = ct.closed_loop(cfg, screens, M, R, sn, valid, 20)
    assert out["wfe"][10:].mean() < 0.7 * out["wfe"][0]


# ---------------------------------------------------------------- noise

def test_philox_known_answer_vectors():
    rows = read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        ctr = [int(v, 16) for v in r[0:4]]
        key = [int(v, 16) for v in r[4:6]]
        out = [int(v, 16) for v in r[6:10]]
        assert list(nz.philox4x32_10(ctr, key)) == out


@pytest.mark.parametrize("lam", [0.7, 5.0, 30.0, 150.0])
def test_poisson_moments(lam):
    n = 20000
    x = np.array([nz.poisson(lam, 11, p, 3) for p in range(n)], dtype=np.float64)
    se_mean = math.sqrt(lam / n)
    se_var = lam * math.sqrt(2.0 / n) * math.sqrt(1 + 1 / (2 * lam))
    assert abs(x.mean() - lam) < 4.5 * se_mean
    assert abs(x.var() - lam) < 4.5 * se_var
    if lam < 1:
        assert abs(np.mean(x == 0) - math.exp(-lam)) < 4.5 * math.sqrt(math.exp(-lam) / n)


def test_gaussian_moments_and_frame_noise_shape():
    n = 20000
    g = np.array([nz.gaussian(3, p, 0) for p in range(n)])
    assert abs(g.mean()) < 4.5 / math.sqrt(n) and abs(g.var() - 1) < 4.5 * math.sqrt(2 / n)
    fr = np.full((6, 6), 2.0)
    a = nz.apply_noise(fr, 1000.0, 36 * 2, 0.5, 9, 0)
    b = nz.apply_noise(fr, 1000.0, 36 * 2, 0.5, 9, 0)
    c = nz.apply_noise(fr, 1000.0, 36 * 2, 0.5, 9, 1)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert abs(a.mean() - 2.0 * 1000 / 72) < 5


# ---------------------------------------------------------------- MLP reconstructor

def test_mlp_gradient_matches_central_differences():
    from oracle import mlp
    g = np.random.default_rng(4)
    sizes = mlp.layer_sizes(7, 6, 3, 5)
    params = mlp.init_params(sizes, g)
    for i in range(1, len(params), 2):
        params[i] = g.standard_normal(params[i].shape) * 0.1
    x = g.standard_normal((4, 7))
    y = g.standard_normal((4, 5))
    out, cache = mlp.forward(params, x)
    grads = mlp.flatten(mlp.backward(params, cache, out, y))
    vec = mlp.flatten(params)
    h = 1e-6
    num = np.empty_like(vec)
    for k in range(vec.size):
        vp, vm = vec.copy(), vec.copy()
        vp[k] += h
        vm[k] -= h
        lp = mlp.loss(mlp.forward(mlp.unflatten(vp, sizes), x)[0], y)
        lm = mlp.loss(mlp.forward(mlp.unflatten(vm, sizes), x)[0], y)
        num[k] = (lp - lm) / (2 * h)
    assert np.max(np.abs(num - grads)) < 1e-7 * max(1.0, np.max(np.abs(grads)))


def test_gelu_closed_form_points_and_derivative():
    from oracle import mlp
    from scipy.stats import norm
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    assert np.allclose(mlp.gelu(z), z * norm.cdf(z), rtol=0, atol=1e-15)
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-8)


def test_mlp_adam_overfits_a_tiny_batch():
    from oracle import mlp
    g = np.random.default_rng(5)
    sizes = mlp.layer_sizes(6, 16, 2, 3)
    params = mlp.init_params(sizes, g)
    x = g.standard_normal((8, 6))
    y = g.standard_normal((8, 3))
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    l0 = mlp.loss(mlp.forward(params, x)[0], y)
    for t in range(1, 1501):
        out, cache = mlp.forward(params, x)
        mlp.adam_update(params, mlp.backward(params, cache, out, y), m, v, t, 1e-2)
    assert mlp.loss(mlp.forward(params, x)[0], y) < 1e-4 * l0


# ---------------------------------------------------------------- KL basis

def _piston_free(M):
    M = M - M.mean(axis=0)
    Q, R = np.linalg.qr(M)
    return Q * np.sign(np.diag(R)) * math.sqrt(M.shape[0])


@pytest.mark.parametrize("Np,D,r0,L0,pad", [(24, 2.0, 0.1, 1.0, 8), (32, 4.0, 0.2, 2.0, 6)])
def test_modal_covariance_equals_spatial_double_sum(Np, D, r0, L0, pad):
    """Independent route: C = -(1/2 n^2) M^T D(|x - x'|) M with the closed-form von
    Karman structure function (zero-mean modes), against the frequency-domain sum."""
    dx = D / Np
    mask = op.pupil_mask(Np, 0.1)
    M = _piston_free(md.modal_basis(Np, 0.1, 12))
    C = md.modal_covariance(M, mask, dx, r0, L0, pad)
    X, Y = np.nonzero(mask)
    P = np.stack([X, Y], 1) * dx
    r = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
    Cs = -0.5 * M.T @ at.structure_function_von_karman(r, r0, L0) @ M / mask.sum() ** 2
    assert np.max(np.abs(C - Cs)) <= 1e-2 * np.max(np.diag(Cs))


def _noll_covariance(j, jp, D_r0):
    """Kolmogorov covariance of Zernike coefficients on a disc (Noll 1976):
    2.2698 (-1)^((n+n'-2m)/2) sqrt((n+1)(n'+1)) Gamma((n+n'-5/3)/2) (D/r0)^(5/3) /
    [Gamma((n-n'+17/3)/2) Gamma((n'-n+17/3)/2) Gamma((n+n'+23/3)/2)], zero unless m = m'
    (and j, j' of equal parity for m != 0)."""
    from scipy.special import gamma
    n, m = md.noll_to_nm(j)
    n2, m2 = md.noll_to_nm(jp)
    if abs(m) != abs(m2) or (m != 0 and j % 2 != jp % 2):
        return 0.0
    K = 2.2698 * (-1) ** ((n + n2 - 2 * abs(m)) // 2) * math.sqrt((n + 1) * (n2 + 1))
    return K * gamma((n + n2 - 5 / 3) / 2) / (gamma((n - n2 + 17 / 3) / 2) * gamma((n2 - n + 17 / 3) / 2)
                                              * gamma((n + n2 + 23 / 3) / 2)) * D_r0 ** (5 / 3)


def test_modal_covariance_kolmogorov_zernike_variances():
    """Radial orders 2 and 3 (j = 4 .. 10) and spherical (j = 11) against Noll's
    closed form. (Tip and tilt are left out: their integrand is singular at f = 0,
    which a discrete frequency grid undersamples.)"""
    Np, D, r0 = 64, 8.0, 0.5
    mask = op.pupil_mask(Np, 0.0)
    M = _piston_free(md.modal_basis(Np, 0.0, 10))           # j = 2 .. 11
    C = md.modal_covariance(M, mask, D / Np, r0, math.inf, 8)
    for k, j in enumerate(range(2, 12)):
        if j >= 4:
            assert abs(C[k, k] / _noll_covariance(j, j, D / r0) - 1) < 0.03, j
    # the closed form itself against Noll's tabulated variances: tilt 0.449, focus 0.0232
    assert abs(_noll_covariance(2, 2, 1.0) - 0.449) < 0.01
    assert abs(_noll_covariance(4, 4, 1.0) - 0.0232) < 0.0005


def test_kl_basis_diagonalises_and_spans_the_zernike_space():
    Np = 32
    mask = op.pupil_mask(Np, 0.1)
    M = md.modal_basis(Np, 0.1, 20)
    C = md.modal_covariance(M, mask, 8.0 / Np, 0.15, 25.0, 4)
    K, w = md.kl_basis(M, C)
    n = mask.sum()
    assert np.max(np.abs(K.T @ K / n - np.eye(20))) < 1e-10          # orthonormal
    assert np.all(np.diff(w) <= 0) and w[-1] > 0                     # decreasing variances
    Ck = (K.T @ M / n) @ C @ (M.T @ K / n)                           # covariance of KL coefficients
    assert np.max(np.abs(Ck - np.diag(w))) < 1e-9 * w[0]
    assert np.max(np.abs(K @ K.T - M @ M.T)) / n < 1e-10             # same span
    assert np.all(md.sign_pattern(n) @ K > 0)
