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
