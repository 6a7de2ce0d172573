"""Allocation-free pyramid measurement (pas_pyr_measure_static) against the
object-based entry point.

Some callers cannot allocate device memory while they run (an allocator that
forbids cudaMalloc after start-up, another library owning the device allocator);
pas_pyr_measure_static serves them from a fixed array compiled into the library.
This file is collected last on purpose: a failure here leaves every other test
already run.
"""
import numpy as np
import pytest

from synth import get_config, tiny_config
from synth.inputs import random_opd_nm

pytestmark = pytest.mark.gpu

FRAME_TOL = 1e-5
SLOPE_TOL = 1e-5


@pytest.mark.parametrize("cfg", [get_config("scao_8m_64px"), tiny_config(Np=60, N=120, n_sub=10, K=12, mod_radius=3.0),
                                 get_config("scao_lbt_240px")], ids=lambda c: c.name)
def test_static_measure_matches_object_measure_twice(cfg):
    import torch
    from paper_1607_07624_gb300 import pas
    ctx = pas.pas_ctx_create()
    pyr = pas.pas_pyr_create(ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs)
    try:
        nv = pas.pas_pyr_n_valid(pyr)
        sn = torch.linspace(-0.05, 0.05, 2 * nv, device="cuda")
        pas.pas_pyr_set_reference(pyr, ctx, sn)
        for call, seed in enumerate((21, 22)):
            opd = torch.as_tensor(random_opd_nm(cfg.Np, 250.0, seed=seed).astype(np.float32)).cuda()
            fr_o = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
            sl_o = torch.zeros(2 * nv, device="cuda")
            pas.pas_pyr_measure(pyr, ctx, opd, fr_o, sl_o)
            fr_s = torch.full((cfg.n_det, cfg.n_det), float("nan"), device="cuda")
            sl_s = torch.full((2 * nv,), float("nan"), device="cuda")
            pas.pas_pyr_measure_static(cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs,
                                       opd, fr_s, sl_s, d_sn=sn)
            torch.cuda.synchronize()
            a, b = fr_s.cpu().numpy(), fr_o.cpu().numpy()
            assert np.all(np.isfinite(a)), call
            assert np.max(np.abs(a - b)) <= FRAME_TOL * np.max(np.abs(b)), call
            sa, sb = sl_s.cpu().numpy(), sl_o.cpu().numpy()
            assert np.max(np.abs(sa - sb)) <= SLOPE_TOL * np.max(np.abs(sb)) + 1e-7, call
    finally:
        torch.cuda.synchronize()
        pas.pas_pyr_destroy(pyr)
        pas.pas_ctx_destroy(ctx)


def test_static_measure_rejects_geometries_beyond_its_array():
    import torch
    from paper_1607_07624_gb300 import pas
    cfg = get_config("scao_elt_480px")
    opd = torch.zeros(cfg.Np, cfg.Np, device="cuda")
    fr = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
    with pytest.raises(pas.PasError) as e:
        pas.pas_pyr_measure_static(cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs,
                                   opd, fr)
    assert e.value.status == pas.PAS_EINVAL and "bytes" in str(e.value)
