"""Batched loops: one graph launch per step drives several independent loops (equal
and different sizes) and reproduces, bit for bit, what each loop does alone."""
import numpy as np
import pytest

from synth import get_config, tiny_config
from synth.configs import with_

pytestmark = pytest.mark.gpu


def _systems():
    from paper_1607_07624_gb300.system import SCAOSystem
    cfg = get_config("scao_8m_64px")
    first = SCAOSystem(cfg, autotune=False, wfe_history=256)
    out = [first]
    for seed in (2001, 2002):
        out.append(SCAOSystem(with_(cfg, seed=seed), basis=first.basis, R=first.R, autotune=False,
                              wfe_history=256))
    small = tiny_config(Np=32, N=64, n_sub=8, K=8, n_modes=20, mod_radius=2.0, S=128)
    out.append(SCAOSystem(small, autotune=False, wfe_history=256))
    return out


def test_batch_steps_reproduce_single_loops():
    import torch
    from paper_1607_07624_gb300 import pas
    systems = _systems()
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
    finally:
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
        assert pas.pas_batch_kernels_per_step(batch) == 5 * 4 + 3
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
