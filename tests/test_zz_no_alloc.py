"""Allocation-free pyramid measurement (pas_pyr_measure_static) against the
object-based entry point.

Some callers cannot allocate device memory while they run (an allocator that
forbids cudaMalloc after start-up, another library owning the device allocator);
pas_pyr_measure_static serves them from a fixed array compiled into the library.
This file is collected last on purpose: a failure here leaves every other test
already run. Besides the object path, the 64 px case is checked against the FP64
oracle directly, and a call on a stream under capture must be refused cleanly.
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


def test_static_measure_matches_the_oracle_on_the_64px_workload():
    import torch
    from oracle import optics as op
    from paper_1607_07624_gb300 import pas
    cfg = get_config("scao_8m_64px")
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    for seed in (31, 32):
        opd = random_opd_nm(cfg.Np, 300.0, seed=seed).astype(np.float32)
        fr = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
        sl = torch.zeros(2 * valid.size, device="cuda")
        pas.pas_pyr_measure_static(cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs,
                                   torch.as_tensor(opd).cuda(), fr, sl)
        torch.cuda.synchronize()
        I = op.pwfs_intensity(opd.astype(np.float64), cfg.wavelength_nm, cfg.obs, cfg.N, cfg.K, cfg.mod_radius)
        fo = op.bin_detector(I, cfg.b)
        so = op.pwfs_slopes(fo, valid, cfg.n_sub)
        assert np.max(np.abs(fr.cpu().numpy() - fo)) <= FRAME_TOL * np.max(fo)
        assert np.max(np.abs(sl.cpu().numpy() - so)) <= SLOPE_TOL * np.max(np.abs(so)) + 1e-7


def test_static_measure_refuses_a_stream_under_capture():
    import torch
    from paper_1607_07624_gb300 import pas
    cfg = tiny_config(Np=32, N=64, n_sub=8, K=8, mod_radius=2.0)
    opd = torch.as_tensor(random_opd_nm(cfg.Np, 150.0, seed=5).astype(np.float32)).cuda()
    fr = torch.zeros(cfg.n_det, cfg.n_det, device="cuda")
    args = (cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius, cfg.wavelength_nm, cfg.obs, opd, fr)
    pas.pas_pyr_measure_static(*args)        # the device's first call: outside any capture
    torch.cuda.synchronize()
    ref = fr.clone()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            with pytest.raises(pas.PasError) as e:
                pas.pas_pyr_measure_static(*args, stream=s)
        finally:
            g.capture_end()
    assert e.value.status == pas.PAS_EINVAL and "captured" in str(e.value)
    # nothing was recorded, and the stream and the entry point still work
    fr.zero_()
    pas.pas_pyr_measure_static(*args, stream=s)
    s.synchronize()
    assert torch.equal(fr, ref)
