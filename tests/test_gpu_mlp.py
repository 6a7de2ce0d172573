"""GPU learned reconstructor against the oracle: the tensor-core GEMM, the
network's single-vector and batched passes, gradients, Adam, training pairs and
its use as the loop's reconstructor."""
import numpy as np
import pytest

from synth import get_config
from synth.inputs import rng

pytestmark = pytest.mark.gpu

FULL = [1424, 1024, 1024, 1024, 400]   # 2 x 712 valid sub-apertures -> 400 modes
SMALL = [416, 256, 256, 100]           # 2 x 208 valid sub-apertures -> 100 modes


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1607_07624_gb300 import pas
    ctx = pas.pas_ctx_create()
    yield torch, pas, ctx
    torch.cuda.synchronize()
    pas.pas_ctx_destroy(ctx)


def bf16_round(x):
    """float -> nearest bfloat16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def make_net(sizes, seed):
    from oracle import mlp as om
    params = om.init_params(sizes, rng(seed))
    g = rng(seed + 1)
    for i in range(1, len(params), 2):
        params[i] = g.standard_normal(params[i].shape) * 0.1
    return [p.astype(np.float32).astype(np.float64) for p in params]


def quantised(params):
    return [bf16_round(p) if p.ndim == 2 else p for p in params]


def net_on_gpu(pas, ctx, sizes, params, max_batch, mean=None, istd=None):
    from oracle import mlp as om
    m = pas.pas_mlp_create(ctx, sizes, max_batch)
    pas.pas_mlp_set_params(m, ctx, om.flatten(params).astype(np.float32))
    if mean is not None:
        pas.pas_mlp_set_norm(m, ctx, mean, istd)
    return m


def slopes_like(n, B, seed):
    g = rng(seed)
    mean = (0.05 * g.standard_normal(n)).astype(np.float32)
    istd = (1.0 / (0.1 + 0.05 * g.random(n))).astype(np.float32)
    S = (mean + g.standard_normal((B, n)) / istd).astype(np.float32)
    return S, mean, istd


# ---------------------------------------------------------------- GEMM

@pytest.mark.parametrize("M,N,K,tile", [(128, 128, 64, 0), (128, 64, 64, 64), (200, 72, 100, 0),
                                        (64, 16, 8, 64), (300, 400, 1024, 256), (1024, 1024, 1424, 0),
                                        (513, 1000, 2000, 128),
                                        # narrow tiles (the batched reconstruction: a few loops)
                                        (400, 8, 1424, 16), (3578, 24, 14312, 32), (300, 5, 72, 16),
                                        # many waves of 128 x 256 tiles in the grouped order (odd row-tile
                                        # count, ragged N)
                                        (4096, 4096, 512, 0), (4224, 4000, 520, 0),
                                        # persistent CTAs (two or more tiles per SM): 128- and
                                        # 256-wide tiles, ragged edges
                                        (4096, 4096, 512, 128), (4000, 4200, 1000, 0)])
def test_gemm_bf16_matches_fp64(env, M, N, K, tile):
    torch, pas, ctx = env
    g = rng(1000 + M + N + K)
    lda = (K + 7) // 8 * 8
    A = torch.zeros(M, lda, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(N, lda, dtype=torch.bfloat16, device="cuda")
    A[:, :K] = torch.as_tensor(g.standard_normal((M, K)).astype(np.float32)).to(torch.bfloat16)
    B[:, :K] = torch.as_tensor(g.standard_normal((N, K)).astype(np.float32)).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    pas.pas_gemm_bf16(ctx, M, N, K, A, lda, B, lda, C, N, err, tile)
    torch.cuda.synchronize()
    assert err.item() == 0
    a = A[:, :K].float().cpu().numpy().astype(np.float64)
    b = B[:, :K].float().cpu().numpy().astype(np.float64)
    ref = a @ b.T
    got = C.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    # float32 accumulation of exact bf16 products
    assert np.all(np.abs(got - ref) <= 1e-5 * (np.abs(a) @ np.abs(b).T) + 1e-30)


def test_gemm_persistent_256_by_256_tiles_match_fp64_on_sampled_rows(env):
    """A product large enough for persistent CTAs with 256 x 256 tiles (ragged in M and
    N: a second 128-row half past the matrix reads zeros): 600 sampled rows against FP64
    with float32 accumulation of exact bf16 products."""
    torch, pas, ctx = env
    g = rng(91)
    M, N, K = 6000, 7000, 320
    A = torch.as_tensor(g.standard_normal((M, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    B = torch.as_tensor(g.standard_normal((N, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    C = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    pas.pas_gemm_bf16(ctx, M, N, K, A, K, B, K, C, N, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    rows = np.unique(np.concatenate([g.integers(0, M, 560), np.arange(M - 40, M)]))
    a = A[torch.as_tensor(rows).cuda()].float().cpu().numpy().astype(np.float64)
    b = B.float().cpu().numpy().astype(np.float64)
    got = C[torch.as_tensor(rows).cuda()].cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - a @ b.T) <= 1e-5 * (np.abs(a) @ np.abs(b).T) + 1e-30)


@pytest.mark.parametrize("M,N,K", [(256, 384, 1024), (4096, 4096, 512), (6000, 7000, 320)])
def test_gemm_wait_that_gives_up_unwinds_and_reports(env, M, N, K):
    """Every pipeline wait of the tensor-core GEMM made to give up at once (wait
    limit 0, a barrier no copy has reached yet): the product-issue and epilogue bits
    are set, the unwinding (copies in flight drained, products completed, tensor
    memory freed) finishes within its own bound, and the context stays usable: the
    same GEMM with the default bound is then exact."""
    torch, pas, ctx = env
    g = rng(77)
    A = torch.as_tensor(g.standard_normal((M, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    B = torch.as_tensor(g.standard_normal((N, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    C = torch.zeros(M, N, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    pas.pas_gemm_bf16_waits(ctx, M, N, K, A, K, B, K, C, N, err, 0)
    torch.cuda.synchronize()
    e = int(err.item())
    assert e & 2 and e & 4, e         # product issue and epilogue gave up
    assert not e & 8, e               # the unwinding completed
    err.zero_()
    C.fill_(float("nan"))
    pas.pas_gemm_bf16(ctx, M, N, K, A, K, B, K, C, N, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    a = A.float().cpu().numpy().astype(np.float64)
    b = B.float().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(C.cpu().numpy() - a @ b.T) <= 1e-5 * (np.abs(a) @ np.abs(b).T))


def test_gemm_rejects_unaligned_leading_dimension(env):
    torch, pas, ctx = env
    A = torch.zeros(128, 100, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(128, 128, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pas.PasError):
        pas.pas_gemm_bf16(ctx, 128, 128, 100, A, 100, A, 100, C, 128, err)


# ---------------------------------------------------------------- network passes

def test_single_vector_inference_matches_oracle(env):
    torch, pas, ctx = env
    from oracle import mlp as om
    params = make_net(FULL, 7)
    S, mean, istd = slopes_like(FULL[0], 3, 8)
    m = net_on_gpu(pas, ctx, FULL, params, 4, mean, istd)
    try:
        q = quantised(params)
        out = torch.zeros(FULL[-1], device="cuda")
        for b in range(3):
            s = torch.as_tensor(S[b]).cuda()
            pas.pas_mlp_apply(m, ctx, s, out)
            torch.cuda.synchronize()
            x = (S[b].astype(np.float64) - mean) * istd
            ref = om.forward(q, x[None, :])[0][0]
            rms = np.sqrt(np.mean(ref ** 2))
            assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-4 * rms
    finally:
        pas.pas_mlp_destroy(m)


@pytest.mark.parametrize("sizes,B", [(FULL, 300), ([37, 50, 23], 70)])
def test_batched_forward_matches_oracle(env, sizes, B):
    torch, pas, ctx = env
    from oracle import mlp as om
    params = make_net(sizes, 9)
    S, mean, istd = slopes_like(sizes[0], B, 10)
    m = net_on_gpu(pas, ctx, sizes, params, 512, mean, istd)
    try:
        out = torch.zeros(B, sizes[-1], device="cuda")
        pas.pas_mlp_forward(m, ctx, B, torch.as_tensor(S).cuda(), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        q = quantised(params)
        x = (S.astype(np.float64) - mean) * istd
        ref = om.forward(q, x)[0]
        rms = np.sqrt(np.mean(ref ** 2))
        # the GEMM operands (inputs, hidden activations) are bf16: loose against FP64
        assert np.sqrt(np.mean((got - ref) ** 2)) <= 1e-2 * rms
        assert np.max(np.abs(got - ref)) <= 5e-2 * rms
        # against the same computation with those roundings applied: closer, though not
        # bitwise (an activation that rounds the other way shifts the whole next layer)
        h = bf16_round(x)
        L = len(q) // 2
        for l in range(L):
            z = h @ q[2 * l].T + q[2 * l + 1]
            h = bf16_round(om.gelu(z)) if l < L - 1 else z
        assert np.sqrt(np.mean((got - h) ** 2)) <= 3e-3 * rms
        assert np.max(np.abs(got - h)) <= 2e-2 * rms
    finally:
        pas.pas_mlp_destroy(m)


@pytest.mark.parametrize("sizes,B", [(FULL, 256), (SMALL, 130), ([37, 50, 23], 70)])
def test_gradients_match_oracle_backward(env, sizes, B):
    torch, pas, ctx = env
    from oracle import mlp as om
    params = make_net(sizes, 11)
    S, mean, istd = slopes_like(sizes[0], B, 12)
    Y = rng(13).standard_normal((B, sizes[-1])).astype(np.float32)
    m = net_on_gpu(pas, ctx, sizes, params, 512, mean, istd)
    try:
        grad = torch.zeros(pas.pas_mlp_n_params(m), device="cuda")
        loss = pas.pas_mlp_gradients(m, ctx, B, torch.as_tensor(S).cuda(), torch.as_tensor(Y).cuda(), grad)
        assert pas.pas_mlp_check(m, ctx) == 0
        q = quantised(params)
        x = (S.astype(np.float64) - mean) * istd
        out, cache = om.forward(q, x)
        ref = om.backward(q, cache, out, Y.astype(np.float64))
        assert abs(loss - om.loss(out, Y)) <= 1e-2 * om.loss(out, Y)
        got = om.unflatten(grad.cpu().numpy().astype(np.float64), sizes)
        for k, (gg, rr) in enumerate(zip(got, ref)):
            rel = np.linalg.norm(gg - rr) / np.linalg.norm(rr)
            cos = np.sum(gg * rr) / (np.linalg.norm(gg) * np.linalg.norm(rr))
            assert rel < 3e-2 and cos > 0.9995, (k, rel, cos)
    finally:
        pas.pas_mlp_destroy(m)


def test_adam_steps_match_oracle_update(env):
    """Two training steps on one batch equal the oracle's Adam fed the same gradients."""
    torch, pas, ctx = env
    from oracle import mlp as om
    sizes, B = SMALL, 128
    params = make_net(sizes, 14)
    S, mean, istd = slopes_like(sizes[0], B, 15)
    Y = rng(16).standard_normal((B, sizes[-1])).astype(np.float32)
    m = net_on_gpu(pas, ctx, sizes, params, B, mean, istd)
    try:
        dS, dY = torch.as_tensor(S).cuda(), torch.as_tensor(Y).cuda()
        idx = torch.arange(B, dtype=torch.int32, device="cuda")
        lr = torch.tensor([1e-3], device="cuda")
        loss = torch.zeros(1, device="cuda")
        grad = torch.zeros(pas.pas_mlp_n_params(m), device="cuda")
        p = [x.copy() for x in params]
        mom = [np.zeros_like(x) for x in params]
        vel = [np.zeros_like(x) for x in params]
        for t in (1, 2):
            pas.pas_mlp_gradients(m, ctx, B, dS, dY, grad)
            g = om.unflatten(grad.cpu().numpy().astype(np.float64), sizes)
            pas.pas_mlp_train(m, ctx, dS, dY, B, B, idx, lr, 1, loss)
            got = om.unflatten(pas.pas_mlp_get_params(m, ctx).astype(np.float64), sizes)
            om.adam_update(p, g, mom, vel, t, 1e-3)
            for k, (gg, rr) in enumerate(zip(got, p)):
                assert np.max(np.abs(gg - rr)) <= 2e-6 * 1e-3 + 1e-6 * np.max(np.abs(rr)), (t, k)
            p = got
        assert pas.pas_mlp_check(m, ctx) == 0
    finally:
        pas.pas_mlp_destroy(m)


def test_training_overfits_a_small_set(env):
    torch, pas, ctx = env
    from oracle import mlp as om
    sizes, n = SMALL, 64
    params = make_net(sizes, 17)
    S, mean, istd = slopes_like(sizes[0], n, 18)
    Y = rng(19).standard_normal((n, sizes[-1])).astype(np.float32)
    m = net_on_gpu(pas, ctx, sizes, params, n, mean, istd)
    try:
        steps = 400
        idx = torch.arange(n, dtype=torch.int32, device="cuda").repeat(steps)
        lr = torch.full((steps,), 1e-3, device="cuda")
        loss = torch.zeros(steps, device="cuda")
        pas.pas_mlp_train(m, ctx, torch.as_tensor(S).cuda(), torch.as_tensor(Y).cuda(), n, n, idx, lr, steps, loss)
        assert pas.pas_mlp_check(m, ctx) == 0
        L = loss.cpu().numpy()
        assert np.all(np.isfinite(L))
        assert L[-1] < 1e-2 * L[0]
        # the loss of step 0 is the oracle's loss of the initial network (bf16 GEMM operands)
        x = (S.astype(np.float64) - mean) * istd
        l0 = om.loss(om.forward(quantised(params), x)[0], Y)
        assert abs(L[0] - l0) <= 1e-2 * l0
    finally:
        pas.pas_mlp_destroy(m)


def test_out_of_range_sample_index_is_reported(env):
    torch, pas, ctx = env
    sizes = [37, 50, 23]
    m = net_on_gpu(pas, ctx, sizes, make_net(sizes, 20), 8)
    try:
        S = torch.zeros(8, 37, device="cuda")
        Y = torch.zeros(8, 23, device="cuda")
        idx = torch.tensor([0, 1, 2, 3, 4, 5, 6, 8], dtype=torch.int32, device="cuda")
        lr = torch.tensor([1e-3], device="cuda")
        loss = torch.zeros(1, device="cuda")
        pas.pas_mlp_train(m, ctx, S, Y, 8, 8, idx, lr, 1, loss)
        with pytest.raises(pas.PasError, match="index"):
            pas.pas_mlp_check(m, ctx)
        assert pas.pas_mlp_check(m, ctx) == 0  # cleared
    finally:
        pas.pas_mlp_destroy(m)


# ---------------------------------------------------------------- data and loop

def test_training_pair_is_pyramid_slopes_and_modal_projection(env):
    torch, pas, ctx = env
    from oracle import modal as md
    cfg = get_config("scao_8m_64px")
    pix = pas.pas_pupil_pixels(cfg.Np, cfg.obs)
    valid = pas.pas_valid_subaps(cfg.Np, cfg.obs, cfg.n_sub)
    M = md.modal_basis(cfg.Np, cfg.obs, cfg.n_modes)
    pyr = pas.pas_pyr_create(ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs, valid)
    dm = pas.pas_dm_create(ctx, M, cfg.Np, cfg.obs)
    try:
        opd = (rng(21).standard_normal((cfg.Np, cfg.Np)) * 40).astype(np.float32)
        d_opd = torch.as_tensor(opd).cuda()
        work = torch.zeros(cfg.Np * cfg.Np + cfg.n_det ** 2, device="cuda")
        s = torch.zeros(2 * valid.size, device="cuda")
        c = torch.zeros(cfg.n_modes, device="cuda")
        pas.pas_mlp_pair(pyr, dm, ctx, d_opd, 2.0, work, s, c)
        frame = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
        s2 = torch.zeros_like(s)
        pas.pas_pyr_measure(pyr, ctx, d_opd * 2.0, frame, s2)
        torch.cuda.synchronize()
        assert torch.equal(s, s2)
        ref = M.T @ (2.0 * opd.astype(np.float64).ravel()[pix]) / pix.size
        assert np.max(np.abs(c.cpu().numpy() - ref)) <= 1e-5 * np.max(np.abs(ref))
    finally:
        pas.pas_pyr_destroy(pyr)
        pas.pas_dm_destroy(dm)


def test_loop_with_single_layer_network_follows_linear_loop(env):
    """A one-layer network W = R, b = 0 reproduces the linear loop up to bf16 rounding of R;
    a non-finite network output is caught and leaves the command finite."""
    torch, pas, ctx = env
    from paper_1607_07624_gb300.system import SCAOSystem
    cfg = get_config("scao_8m_64px")
    sys_lin = SCAOSystem(cfg, autotune=False)
    try:
        sys_lin.step(40)
        w_lin = sys_lin.wfe_nm(40)
        sys_lin.set_state(0, np.zeros((sys_lin.delay, sys_lin.n_modes), np.float32))
        R = sys_lin.R.astype(np.float64)
        sizes = [R.shape[1], R.shape[0]]
        m = pas.pas_mlp_create(sys_lin.ctx, sizes, 1)
        try:
            pas.pas_mlp_set_params(m, sys_lin.ctx, np.concatenate([R.ravel(), np.zeros(R.shape[0])]).astype(np.float32))
            pas.pas_loop_set_mlp(sys_lin.loop, sys_lin.ctx, m)
            sys_lin.step(40)
            w_mlp = sys_lin.wfe_nm(40)
            assert pas.pas_mlp_check(m, sys_lin.ctx) == 0
            assert np.all(np.abs(w_mlp - w_lin) <= 0.01 * w_lin + 0.05)
            # poison one weight: that coefficient's update becomes 0, the fault is reported
            bad = np.concatenate([R.ravel(), np.zeros(R.shape[0])]).astype(np.float32)
            bad[5 * R.shape[1]] = np.inf
            pas.pas_mlp_set_params(m, sys_lin.ctx, bad)
            sys_lin.step(3)
            assert pas.pas_mlp_check(m, sys_lin.ctx) == 1
            torch.cuda.synchronize()
            assert torch.isfinite(sys_lin.loop_cmd).all()
            # back to the linear reconstructor
            pas.pas_loop_set_mlp(sys_lin.loop, sys_lin.ctx, None)
            sys_lin.step(3)
            assert pas.pas_mlp_check(m, sys_lin.ctx) == 0
        finally:
            pas.pas_mlp_destroy(m)
    finally:
        sys_lin.close()
