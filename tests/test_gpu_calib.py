"""GPU calibration: FP64 Jacobi-SVD pseudo-inverse, FP64 products and the Cholesky-QR
Zernike basis against NumPy's SVD, the oracle's pseudo-inverse and Gram-Schmidt."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1607_07624_gb300 import pas
    ctx = pas.pas_ctx_create()
    yield torch, pas, ctx
    torch.cuda.synchronize()
    pas.pas_ctx_destroy(ctx)


def _gpu_pinv(torch, pas, ctx, A, rcond):
    m, n = A.shape
    d_A = torch.as_tensor(np.ascontiguousarray(A.T)).cuda()      # column-major m x n
    d_P = torch.empty(n, m, dtype=torch.float64, device="cuda")
    sv, rank, sweeps = pas.pas_pinv_f64(ctx, d_A, m, n, rcond, d_P)
    return d_P.cpu().numpy(), sv, rank, sweeps


def test_pinv_matches_the_oracle_on_the_64px_interaction_matrix(env):
    torch, pas, ctx = env
    from oracle import modal as md
    from oracle import optics as op
    from synth import get_config
    cfg = get_config("scao_8m_64px")
    M = md.modal_basis(cfg.Np, cfg.obs, cfg.n_modes)
    mask = op.pupil_mask(cfg.Np, cfg.obs)
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    _, sn = op.pwfs_measure(np.zeros((cfg.Np, cfg.Np)), cfg, valid)
    IM = md.interaction_matrix(lambda o: op.pwfs_measure(o, cfg, valid, sn)[1], M, mask, cfg.pushpull_nm)
    P, sv, rank, sweeps = _gpu_pinv(torch, pas, ctx, IM, 1e-3)
    R = md.pseudo_inverse(IM, 1e-3)
    assert np.max(np.abs(P - R)) <= 1e-10 * np.max(np.abs(R))
    s_ref = np.linalg.svd(IM, compute_uv=False)
    assert np.max(np.abs(sv - s_ref)) <= 1e-12 * s_ref[0]
    assert rank == np.sum(s_ref >= 1e-3 * s_ref[0]) and 1 <= sweeps <= 30


@pytest.mark.parametrize("m,n", [(300, 120), (257, 81), (64, 64), (1424, 400)])
def test_pinv_truncates_small_singular_values_like_numpy(env, m, n):
    torch, pas, ctx = env
    g = np.random.default_rng(m + n)
    U, _ = np.linalg.qr(g.standard_normal((m, n)))
    V, _ = np.linalg.qr(g.standard_normal((n, n)))
    s = np.logspace(0, -2.5, n)
    s[-n // 6:] *= 1e-4          # a block well below rcond
    A = (U * s) @ V.T
    P, sv, rank, _ = _gpu_pinv(torch, pas, ctx, A, 1e-3)
    Us, ss, Vt = np.linalg.svd(A, full_matrices=False)
    keep = ss >= 1e-3 * ss[0]
    R = (Vt[keep].T / ss[keep]) @ Us[:, keep].T
    assert rank == int(keep.sum())
    assert np.max(np.abs(sv - ss)) <= 1e-12 * ss[0]
    assert np.max(np.abs(P - R)) <= 1e-9 * np.max(np.abs(R))
    # full rank: P A = I
    if keep.all():
        assert np.max(np.abs(P @ A - np.eye(n))) < 1e-10


def test_gemm_f64_strided_forms(env):
    torch, pas, ctx = env
    g = np.random.default_rng(3)
    m, n = 531, 70
    Z = g.standard_normal((m, n))
    T = g.standard_normal((n, n))
    w = g.random(n)
    Zd = torch.as_tensor(np.ascontiguousarray(Z.T)).cuda()
    Td = torch.as_tensor(T).cuda()
    wd = torch.as_tensor(w).cuda()
    G = torch.empty(n, n, dtype=torch.float64, device="cuda")
    pas.pas_gemm_f64(ctx, Zd, m, 1, Zd, m, 1, None, n, n, m, G, n)            # Z^T Z
    Q = torch.empty(n, m, dtype=torch.float64, device="cuda")
    pas.pas_gemm_f64(ctx, Td, 1, n, Zd, 1, m, wd, n, m, n, Q, m)              # (Z diag(w) T)^T
    torch.cuda.synchronize()
    assert np.max(np.abs(G.cpu().numpy() - Z.T @ Z)) < 1e-11 * np.abs(Z.T @ Z).max()
    ref = ((Z * w) @ T).T
    assert np.max(np.abs(Q.cpu().numpy() - ref)) < 1e-11 * np.abs(ref).max()


def test_cholesky_qr_zernike_basis_equals_gram_schmidt(env):
    torch, pas, ctx = env
    from oracle import modal as md
    from paper_1607_07624_gb300 import calib
    Np, obs, n = 64, 0.1, 100
    pix = pas.pas_pupil_pixels(Np, obs)
    Q = calib.zernike_basis_gpu(ctx, Np, pix, n)
    assert np.max(np.abs(Q - calib.zernike_basis(Np, pix, n))) < 1e-9
    assert np.max(np.abs(Q - md.modal_basis(Np, obs, n))) < 1e-9
    assert np.max(np.abs(Q.T @ Q / pix.size - np.eye(n))) < 1e-12


def test_interaction_matrix_kernel_against_the_oracle_measurements(env):
    """pas_calib_interaction_matrix on the 64 px workload (bf16 DM basis included:
    the push reads the DM's own basis) against the oracle's push-pull matrix."""
    torch, pas, ctx = env
    from oracle import modal as md
    from oracle import optics as op
    from synth import get_config
    cfg = get_config("scao_8m_64px")
    M = md.modal_basis(cfg.Np, cfg.obs, 30)
    mask = op.pupil_mask(cfg.Np, cfg.obs)
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    _, sn = op.pwfs_measure(np.zeros((cfg.Np, cfg.Np)), cfg, valid)
    IM = md.interaction_matrix(lambda o: op.pwfs_measure(o, cfg, valid, sn)[1], M, mask, cfg.pushpull_nm)
    pyr = pas.pas_pyr_create(ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs)
    try:
        for prec, tol in ((pas.PAS_FP32, 1e-4), (pas.PAS_BF16, 2e-2)):
            dm = pas.pas_dm_create(ctx, M.astype(np.float32), cfg.Np, cfg.obs, prec)
            try:
                d = torch.empty(M.shape[1], 2 * valid.size, dtype=torch.float64, device="cuda")
                # a noise setting must not reach the calibration
                pas.pas_pyr_set_noise(pyr, ctx, 1e5, 0.5, 7, 0)
                pas.pas_calib_interaction_matrix(ctx, dm, d, cfg.pushpull_nm, M.shape[1], 2 * valid.size, pyr=pyr)
                pas.pas_pyr_set_noise(pyr, ctx, 0.0, 0.0, 0, 0)
                g = d.t().cpu().numpy()
                assert np.max(np.abs(g - IM)) <= tol * np.max(np.abs(IM)), prec
            finally:
                pas.pas_dm_destroy(dm)
    finally:
        pas.pas_pyr_destroy(pyr)
