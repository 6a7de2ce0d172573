"""Batched loops: one graph launch per step drives several independent loops (equal
and different sizes) and reproduces, bit for bit, what each loop does alone."""
import numpy as np
import pytest

from synth import get_config, tiny_config
from synth.configs import with_

pytestmark = pytest.mark.gpu


def _systems(share_dm=True):
    """Three realisations of the 64 px system (sharing one DM object unless share_dm is
    false) and a smaller loop."""
    from paper_1607_07624_gb300.system import SCAOSystem
    cfg = get_config("scao_8m_64px")
    first = SCAOSystem(cfg, autotune=False, wfe_history=256)
    out = [first]
    for seed in (2001, 2002):
        out.append(SCAOSystem(with_(cfg, seed=seed), basis=first.basis, R=first.R, autotune=False,
                              wfe_history=256, dm=first.dm if share_dm else None))
    small = tiny_config(Np=32, N=64, n_sub=8, K=8, n_modes=20, mod_radius=2.0, S=128)
    out.append(SCAOSystem(small, autotune=False, wfe_history=256))
    return out


@pytest.mark.parametrize("share_dm", [False, True])
def test_batch_steps_reproduce_single_loops(share_dm):
    import torch
    from paper_1607_07624_gb300 import pas
    systems = _systems(share_dm)
    batch = None
    try:
        n = 40
        ref = []
        for s in systems:
            s.step(n)
            ref.append(s.wfe_nm(n))
            s.set_state(0, np.zeros((s.delay, s.n_modes), np.float32))
        ctx = systems[0].ctx
        batch = pas.pas_batch_create(ctx, [s.loop for s in systems])
        assert pas.pas_batch_size(batch) == len(systems)
        assert pas.pas_batch_n_residual_groups(batch) == (1 if share_dm else 0)
        pas.pas_batch_step(batch, ctx, n)
        torch.cuda.synchronize()
        for s, r in zip(systems, ref):
            st, _ = pas.pas_loop_step(s.loop, s.ctx, 0, stats=True)
            assert st == n
            assert np.array_equal(s.wfe_nm(n), r)
        # realisations differ (different screens), the batch does not mix them
        assert not np.array_equal(ref[0], ref[1])
    finally:
        if batch is not None:
            pas.pas_batch_destroy(batch)
        for s in systems:
            s.close()


def test_batch_rejects_duplicates_and_null():
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    s = SCAOSystem(tiny_config(Np=16, N=32, n_sub=4, K=4, n_modes=8, S=64), autotune=False, wfe_history=16)
    try:
        with pytest.raises(pas.PasError, match="twice"):
            pas.pas_batch_create(s.ctx, [s.loop, s.loop])
        with pytest.raises(pas.PasError):
            pas.pas_batch_create(s.ctx, [])
        # a second loop on the same pyramid object: the sensors' intermediates would race
        other = pas.pas_loop_create(s.ctx, s.atmo, s.pyr, s.rec, s.dm, s.d_gain, 1, 16)
        try:
            with pytest.raises(pas.PasError, match="sensor"):
                pas.pas_batch_create(s.ctx, [s.loop, other])
            with pytest.raises(pas.PasError, match="flag"):
                pas.pas_batch_create_ex(s.ctx, [s.loop], 2)
        finally:
            pas.pas_loop_destroy(other)
    finally:
        s.close()


def test_a_loop_held_by_a_batch_cannot_be_reconfigured():
    """The batch's graph holds its loops' steps as captured: re-configuring a member
    (integrating detector, camera, network) is refused until the batch is gone."""
    import torch
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    s = SCAOSystem(tiny_config(Np=48, N=96, n_sub=8, K=8, n_modes=20, mod_radius=2.0, S=128), autotune=False,
                   wfe_history=16)
    psf = pas.pas_psf_create(s.ctx, 48, 2, 1650.0, s.cfg.obs)
    try:
        acc = torch.zeros(96, 96, device="cuda")
        b1 = pas.pas_batch_create(s.ctx, [s.loop])
        b2 = pas.pas_batch_create(s.ctx, [s.loop])
        for b in (b1, b2):
            with pytest.raises(pas.PasError, match="batch"):
                pas.pas_loop_set_integration(s.loop, s.ctx, 2)
            with pytest.raises(pas.PasError, match="batch"):
                pas.pas_loop_attach_camera(s.loop, s.ctx, psf, acc)
            pas.pas_batch_destroy(b)
        pas.pas_loop_set_integration(s.loop, s.ctx, 2)
        pas.pas_loop_attach_camera(s.loop, s.ctx, psf, acc)
        pas.pas_loop_step(s.loop, s.ctx, 3)
        torch.cuda.synchronize()
        pas.pas_loop_attach_camera(s.loop, s.ctx, None)
    finally:
        pas.pas_psf_destroy(psf)
        s.close()


def test_loops_sharing_a_bf16_reconstructor_get_one_tensor_core_product():
    """Five realisations of the 64 px workload share one bf16 reconstructor object: the
    batch reconstructs them with one tensor-core product (R S^T, float32 accumulation)
    and the integrator in its epilogue. After one step each loop's modal update equals
    R s for its own slopes (FP64, the bf16 reconstructor's rounding: 1 % of the RMS),
    and over 40 steps the loops follow the same loops stepped alone with their own
    bf16 matrix-vector product (per-step WFE within 1 nm)."""
    import torch
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    cfg = with_(get_config("scao_8m_64px"), K=24)   # the 64 px optics in their settling setting
    first = SCAOSystem(cfg, autotune=False, wfe_history=64, recon_precision=pas.PAS_BF16)
    systems, alone, batch = [first], [], None
    try:
        for seed in (2001, 2002, 2003, 2004):
            systems.append(SCAOSystem(with_(cfg, seed=seed), basis=first.basis, R=first.R, rec=first.rec,
                                      autotune=False, wfe_history=64))
        for s in systems:   # the same loops, each with a reconstructor of its own
            alone.append(SCAOSystem(s.cfg, basis=first.basis, R=first.R, recon_precision=pas.PAS_BF16,
                                    autotune=False, wfe_history=64))
        ctx = first.ctx
        batch = pas.pas_batch_create(ctx, [s.loop for s in systems])
        assert pas.pas_batch_n_groups(batch) == 1
        # one row tile of R: the product splits its reduction (partials, then the integrator)
        assert pas.pas_batch_kernels_per_step(batch) == 5 * 4 + 4
        pas.pas_batch_step(batch, ctx, 1)
        torch.cuda.synchronize()
        assert pas.pas_batch_check(batch, ctx) == 0
        R = first.R.astype(np.float64)
        for s in systems:
            st, _ = pas.pas_loop_step(s.loop, s.ctx, 0, stats=True)
            assert st == 1
            ref = R @ s.loop_slopes.cpu().numpy().astype(np.float64)
            got = s.loop_dmodes.cpu().numpy().astype(np.float64)
            assert np.sqrt(np.mean((got - ref) ** 2)) <= 0.01 * np.sqrt(np.mean(ref ** 2))
            # the integrator: command = gain x update after one step from zero
            assert np.allclose(s.loop_cmd.cpu().numpy(), cfg.gain * s.loop_dmodes.cpu().numpy(), rtol=1e-6,
                               atol=1e-6)
        pas.pas_batch_step(batch, ctx, 39)
        torch.cuda.synchronize()
        for s, a in zip(systems, alone):
            a.step(40)
            assert np.max(np.abs(s.wfe_nm(40) - a.wfe_nm(40))) <= 1.0
    finally:
        if batch is not None:
            pas.pas_batch_destroy(batch)
        for s in alone + systems[1:] + systems[:1]:
            s.close()


def test_loops_sharing_a_network_get_one_batched_forward():
    """Four realisations of the 64 px workload share one network (one layer W = R, b = 0,
    the linear reconstructor as a network): the batch runs one batched forward through the
    tensor-core layers per step (bf16 inputs and activations) and each loop's integrator on
    its output. After one step each loop's update equals R s (1 % of the RMS: the bf16
    rounding of inputs and weights); over 40 steps the loops follow the same loops stepped
    alone with their own single-vector chains (per-step WFE within 2 nm). More loops than
    the network's batch size are refused."""
    import torch
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    cfg = with_(get_config("scao_8m_64px"), K=24)
    first = SCAOSystem(cfg, autotune=False, wfe_history=64)
    R = first.R.astype(np.float64)
    params = np.concatenate([R.ravel(), np.zeros(R.shape[0])]).astype(np.float32)
    sizes = [R.shape[1], R.shape[0]]
    systems, alone, nets, batch = [first], [], [], None
    try:
        for seed in (2001, 2002, 2003):
            systems.append(SCAOSystem(with_(cfg, seed=seed), basis=first.basis, R=first.R, autotune=False,
                                      wfe_history=64))
        shared = pas.pas_mlp_create(first.ctx, sizes, 4)
        nets.append(shared)
        pas.pas_mlp_set_params(shared, first.ctx, params)
        for s in systems:
            pas.pas_loop_set_mlp(s.loop, s.ctx, shared)
            a = SCAOSystem(s.cfg, basis=first.basis, R=first.R, autotune=False, wfe_history=64)
            own = pas.pas_mlp_create(a.ctx, sizes, 1)
            nets.append(own)
            pas.pas_mlp_set_params(own, a.ctx, params)
            pas.pas_loop_set_mlp(a.loop, a.ctx, own)
            alone.append(a)
        ctx = first.ctx
        batch = pas.pas_batch_create(ctx, [s.loop for s in systems])
        assert pas.pas_batch_n_groups(batch) == 1
        # gather, the layer's product split over K and its finishing sum, integrators, counters
        assert pas.pas_batch_kernels_per_step(batch) == 4 * 4 + (1 + 2 + 2)
        pas.pas_batch_step(batch, ctx, 1)
        torch.cuda.synchronize()
        assert pas.pas_batch_check(batch, ctx) == 0
        for s in systems:
            st, _ = pas.pas_loop_step(s.loop, s.ctx, 0, stats=True)
            assert st == 1
            ref = R @ s.loop_slopes.cpu().numpy().astype(np.float64)
            got = s.loop_dmodes.cpu().numpy().astype(np.float64)
            assert np.sqrt(np.mean((got - ref) ** 2)) <= 0.01 * np.sqrt(np.mean(ref ** 2))
            assert np.allclose(s.loop_cmd.cpu().numpy(), cfg.gain * s.loop_dmodes.cpu().numpy(), rtol=1e-6,
                               atol=1e-6)
        pas.pas_batch_step(batch, ctx, 39)
        torch.cuda.synchronize()
        assert pas.pas_mlp_check(shared, ctx) == 0
        for s, a in zip(systems, alone):
            a.step(40)
            assert np.max(np.abs(s.wfe_nm(40) - a.wfe_nm(40))) <= 2.0
        pas.pas_batch_destroy(batch)
        batch = None
        # a fifth loop on the same network: more than its batch size of 4
        extra = SCAOSystem(with_(cfg, seed=2004), basis=first.basis, R=first.R, autotune=False, wfe_history=64)
        try:
            pas.pas_loop_set_mlp(extra.loop, extra.ctx, shared)
            with pytest.raises(pas.PasError, match="share a network"):
                pas.pas_batch_create(ctx, [s.loop for s in systems] + [extra.loop])
            pas.pas_loop_set_mlp(extra.loop, extra.ctx, None)
        finally:
            extra.close()
    finally:
        if batch is not None:
            pas.pas_batch_destroy(batch)
        for s in alone + systems:
            pas.pas_loop_set_mlp(s.loop, s.ctx, None)
        for m in nets:
            pas.pas_mlp_destroy(m)
        for s in alone + systems[1:] + systems[:1]:
            s.close()


def _mixed_systems():
    """Pyramid loops of two transform lengths (one with an integrating detector) and a
    Shack-Hartmann loop."""
    from paper_1607_07624_gb300.system import SCAOSystem
    out = _systems()
    small = tiny_config(Np=32, N=64, n_sub=8, K=8, n_modes=20, mod_radius=2.0, S=128)
    out.append(SCAOSystem(with_(small, seed=77), autotune=False, wfe_history=256, detector_steps=2))
    out.append(SCAOSystem(with_(small, seed=78), autotune=False, wfe_history=256, sensor="sh"))
    return out


def _run_alone(systems, n):
    ref = []
    for s in systems:
        s.step(n)
        ref.append((s.wfe_nm(n), s.loop_cmd.cpu().numpy().copy()))
        s.set_state(0, np.zeros((s.delay, s.n_modes), np.float32))
    return ref


def test_persistent_batch_reproduces_single_loops():
    """One persistent launch per transform length runs every pyramid loop's rows and
    columns passes from one task queue; each loop's WFE history and command equal
    those of the loop stepped alone, bit for bit."""
    import torch
    from paper_1607_07624_gb300 import pas
    systems = _mixed_systems()
    batch = None
    try:
        n = 40
        ref = _run_alone(systems, n)
        ctx = systems[0].ctx
        batch = pas.pas_batch_create_ex(ctx, [s.loop for s in systems], pas.PAS_BATCH_PERSISTENT)
        assert pas.pas_batch_n_persistent(batch) == 2          # N = 128 and N = 64
        geo = [pas.pas_batch_persistent_geometry(batch, ctx, g) for g in range(2)]
        assert sorted(g_["N"] for g_ in geo) == [64, 128]
        for g_ in geo:
            assert g_["threads"] % 32 == 0 and g_["ctas"] >= 1 and g_["columns_tasks"] > 0
            assert g_["rows_per_task"] in (1, 2, 4, 8) and g_["rows_per_task"] * 32 <= g_["threads"]
        # 5 pyramid loops: residual + slopes + reconstruction; the SH loop whole (3); the
        # three loops sharing a DM: one gather and one residual kernel in place of 3
        assert pas.pas_batch_n_residual_groups(batch) == 1
        assert pas.pas_batch_kernels_per_step(batch) == 5 * 3 + 3 + 2 - 3 + 2
        pas.pas_batch_step(batch, ctx, n)
        torch.cuda.synchronize()
        assert pas.pas_batch_check(batch, ctx) == 0
        for s, (w, c) in zip(systems, ref):
            st, _ = pas.pas_loop_step(s.loop, s.ctx, 0, stats=True)
            assert st == n
            assert np.array_equal(s.wfe_nm(n), w)
            assert np.array_equal(s.loop_cmd.cpu().numpy(), c)
    finally:
        if batch is not None:
            pas.pas_batch_destroy(batch)
        for s in systems:
            s.close()


def test_persistent_batch_wait_runs_out_and_the_context_stays_usable():
    """With the rows pass withheld every columns task waits for a count that nothing
    advances: the bounded wait gives up (limit 0 and 64 polls), the launch completes,
    PAS_ETIMEOUT is reported once, and the batch then steps as before."""
    import torch
    from paper_1607_07624_gb300 import pas
    systems = _systems()
    batch = None
    try:
        n = 12
        ref = _run_alone(systems, n)
        ctx = systems[0].ctx
        batch = pas.pas_batch_create_ex(ctx, [s.loop for s in systems], pas.PAS_BATCH_PERSISTENT)
        for limit in (0, 64):
            pas.pas_batch_set_wait_limit(batch, ctx, limit)
            st, fault = pas.pas_batch_probe_waits(batch)
            assert st == pas.PAS_ETIMEOUT and fault & 0x100
            assert pas.pas_batch_check(batch, ctx) == 0       # reported once
        with pytest.raises(pas.PasError):
            pas.pas_batch_set_wait_limit(batch, ctx, -1)
        pas.pas_batch_set_wait_limit(batch, ctx, 1 << 21)
        for s in systems:   # the probe left the loops' states as they were
            st, _ = pas.pas_loop_step(s.loop, s.ctx, 0, stats=True)
            assert st == 0
        pas.pas_batch_step(batch, ctx, n)
        torch.cuda.synchronize()
        assert pas.pas_batch_check(batch, ctx) == 0
        for s, (w, c) in zip(systems, ref):
            assert np.array_equal(s.wfe_nm(n), w)
            assert np.array_equal(s.loop_cmd.cpu().numpy(), c)
    finally:
        if batch is not None:
            pas.pas_batch_destroy(batch)
        for s in systems:
            s.close()


def test_persistent_batch_with_shared_bf16_reconstructor_matches_graph_branches():
    """Persistent pyramid launch and tensor-core group reconstruction together give
    the same commands as the batch of graph branches, bit for bit."""
    import torch
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    cfg = get_config("scao_8m_64px")
    first = SCAOSystem(cfg, autotune=False, wfe_history=64, recon_precision=pas.PAS_BF16)
    systems, batches = [first], []
    try:
        for seed in (2001, 2002, 2003):
            systems.append(SCAOSystem(with_(cfg, seed=seed), basis=first.basis, R=first.R, rec=first.rec,
                                      autotune=False, wfe_history=64))
        ctx = first.ctx
        out = []
        for flags in (0, pas.PAS_BATCH_PERSISTENT):
            b = pas.pas_batch_create_ex(ctx, [s.loop for s in systems], flags)
            batches.append(b)
            assert pas.pas_batch_n_groups(b) == 1
            pas.pas_batch_step(b, ctx, 30)
            torch.cuda.synchronize()
            assert pas.pas_batch_check(b, ctx) == 0
            out.append([(s.wfe_nm(30), s.loop_cmd.cpu().numpy().copy()) for s in systems])
            for s in systems:
                s.set_state(0, np.zeros((s.delay, s.n_modes), np.float32))
            pas.pas_batch_destroy(b)
            batches.pop()
        for (w0, c0), (w1, c1) in zip(*out):
            assert np.array_equal(w0, w1) and np.array_equal(c0, c1)
    finally:
        for b in batches:
            pas.pas_batch_destroy(b)
        for s in systems[1:] + systems[:1]:
            s.close()


@pytest.mark.parametrize("precision,n_loops", [("fp32", 9), ("bf16", 5)])
def test_shared_dm_residual_batches_reproduce_single_loops(precision, n_loops):
    """Loops sharing one DM object get their residuals from one basis pass (8 loops per
    CTA for a float32 basis, 4 for bf16: a partial last chunk here). An off-axis loop
    joins the group; a source at finite height keeps its own residual kernel. Every
    loop's WFE history and command equal those of the loop stepped alone."""
    import torch
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    cfg = with_(get_config("scao_8m_64px"), n_steps=20)
    prec = pas.PAS_BF16 if precision == "bf16" else pas.PAS_FP32
    first = SCAOSystem(cfg, autotune=False, wfe_history=64, dm_precision=prec)
    systems, batch = [first], None
    try:
        for i in range(1, n_loops):
            source = (2.0, 30.0) if i == 1 else (1.0, 60.0, 90e3) if i == 2 else None
            systems.append(SCAOSystem(with_(cfg, seed=3000 + i), basis=first.basis, R=first.R, dm=first.dm,
                                      autotune=False, wfe_history=64, source=source))
        n = 20
        ref = _run_alone(systems, n)
        ctx = first.ctx
        batch = pas.pas_batch_create(ctx, [s.loop for s in systems])
        assert pas.pas_batch_n_residual_groups(batch) == 1
        pas.pas_batch_step(batch, ctx, n)
        torch.cuda.synchronize()
        for s, (w, c) in zip(systems, ref):
            assert np.array_equal(s.wfe_nm(n), w)
            assert np.array_equal(s.loop_cmd.cpu().numpy(), c)
    finally:
        if batch is not None:
            pas.pas_batch_destroy(batch)
        for s in systems[1:] + systems[:1]:
            s.close()
