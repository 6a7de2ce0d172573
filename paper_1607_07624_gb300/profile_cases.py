"""Short, seeded runs of one workload's loop for a profiler (ncu): the loop of a workload's
shape with a seeded random basis and reconstructor of the right sizes (no calibration), a
fixed pyramid launch geometry, a few steps through the loop's CUDA graph. Timing only: the
wavefront error of a random system means nothing.

    python -m paper_1607_07624_gb300.profile_cases scao_elt_480px --basis fp32 --steps 4
    python -m paper_1607_07624_gb300.profile_cases scao_8m_64px --batch 16 --persistent
    python -m paper_1607_07624_gb300.profile_cases gemm --gemm 8192 --steps 3
    python -m paper_1607_07624_gb300.profile_cases psf --psf 240,8 --steps 4
    python -m paper_1607_07624_gb300.profile_cases mlp --mlp 1424,1024,1024,1024,400 --steps 20

Kernel launches: with --batch 0 every step launches the loop's kernels once, in step order
(residual, rows pass, columns pass, slopes, reconstructor), so ``ncu -k regex:<kernel> -s
<steps before> -c 1`` selects one step's launch. --profile-graph also runs the loop's
profiling graph once per step after the plain steps (events between the kernels).
"""
import argparse

import torch

from . import pas
from .system import SCAOSystem

_PREC = {"fp32": pas.PAS_FP32, "bf16": pas.PAS_BF16}
_TAPS = {"auto": pas.PAS_TAPS_AUTO, "tma": pas.PAS_TAPS_TMA, "copy": pas.PAS_TAPS_COPY}


def _random_system(cfg, basis_prec, recon_prec, tuning, seed, dm=None, rec=None, basis=None, R=None):
    if basis is None:
        gen = torch.Generator(device="cuda").manual_seed(seed)
        pix = pas.pas_pupil_pixels(cfg.Np, cfg.obs)
        valid = pas.pas_valid_subaps(cfg.Np, cfg.obs, cfg.n_sub)
        basis = torch.randn(pix.size, cfg.n_modes, device="cuda", generator=gen).cpu().numpy()
        R = (torch.randn(cfg.n_modes, 2 * valid.size, device="cuda", generator=gen) * 1e-3).cpu().numpy()
    return SCAOSystem(cfg, basis=basis, R=R, dm=dm, rec=rec, dm_precision=basis_prec, recon_precision=recon_prec,
                      autotune=tuning, build_loop=False, wfe_history=64)


def _gemm(n, steps, seed):
    ctx = pas.pas_ctx_create(torch.cuda.current_stream())
    try:
        gen = torch.Generator(device="cuda").manual_seed(seed)
        A = torch.randn(n, n, device="cuda", generator=gen).to(torch.bfloat16)
        B = torch.randn(n, n, device="cuda", generator=gen).to(torch.bfloat16)
        C = torch.empty(n, n, device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        for _ in range(steps):
            pas.pas_gemm_bf16(ctx, n, n, n, A, n, B, n, C, n, err)
        torch.cuda.synchronize()
        print(f"gemm {n}^3 x {steps}: error word {int(err.item())}")
        return 0 if int(err.item()) == 0 else 1
    finally:
        pas.pas_ctx_destroy(ctx)


def _psf(spec, steps, seed):
    """--steps integrated PSF frames (1650 nm) of a seeded 150 nm RMS residual."""
    import numpy as np
    from synth.inputs import random_opd_nm
    Np, nd = (int(x) for x in spec.split(","))
    ctx = pas.pas_ctx_create(torch.cuda.current_stream())
    h = pas.pas_psf_create(ctx, Np, nd, 1650.0, 0.1)
    try:
        N = pas.pas_psf_size(h)
        opd = torch.as_tensor(random_opd_nm(Np, 150.0, seed=seed).astype(np.float32)).cuda()
        acc = torch.zeros(N, N, device="cuda")
        sr = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(steps):
            pas.pas_psf_compute(h, ctx, opd, acc, True, sr)
        torch.cuda.synchronize()
        print(f"psf {N}x{N} x {steps}: Strehl {float(sr.item()):.4f}")
        return 0
    finally:
        pas.pas_psf_destroy(h)
        pas.pas_ctx_destroy(ctx)


def _mlp(spec, batch, steps, seed):
    """--steps Adam steps (one captured graph replay each, after 5 that capture it) of the
    learned reconstructor with layer sizes `spec` on a seeded normal data set of 65536
    pairs, batch `batch`."""
    from .learned import MLPReconstructor
    sizes = [int(x) for x in spec.split(",")]
    ctx = pas.pas_ctx_create(torch.cuda.current_stream())
    mlp = None
    try:
        mlp = MLPReconstructor(ctx, sizes, max_batch=batch, seed=seed)
        gen = torch.Generator(device="cuda").manual_seed(seed)
        n_data = 65536
        S = torch.randn(n_data, sizes[0], device="cuda", generator=gen)
        Y = torch.randn(n_data, sizes[-1], device="cuda", generator=gen)
        idx = torch.randint(0, n_data, (max(steps, 5) * batch,), device="cuda", generator=gen, dtype=torch.int32)
        lr = torch.full((max(steps, 5),), 1e-4, device="cuda")
        loss = torch.zeros(max(steps, 5), device="cuda")
        pas.pas_mlp_train(mlp.h, ctx, S, Y, n_data, batch, idx, lr, 5, loss)
        pas.pas_mlp_train(mlp.h, ctx, S, Y, n_data, batch, idx, lr, steps, loss)
        torch.cuda.synchronize()
        pas.pas_mlp_check(mlp.h, ctx)
        print(f"mlp {sizes} batch {batch} x {steps} steps: last loss {float(loss[steps - 1].item()):.4f}")
        return 0
    finally:
        if mlp is not None:
            mlp.close()
        pas.pas_ctx_destroy(ctx)


def main(argv=None):
    from synth import get_config
    from synth.configs import with_
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("workload", help="scao_8m_64px, scao_lbt_240px or scao_elt_480px (or gemm with --gemm, "
                    "psf with --psf, mlp with --mlp)")
    ap.add_argument("--gemm", type=int, default=0, help="instead of a loop: --steps tensor-core products "
                    "C = A B^T of n x n bf16 matrices (seeded normal entries), float32 C")
    ap.add_argument("--psf", default="", help="instead of a loop: --steps integrated frames of the PSF camera "
                    "for pupil,padding (e.g. 240,8)")
    ap.add_argument("--mlp", default="", help="instead of a loop: --steps training steps of the learned "
                    "reconstructor with these layer sizes (e.g. 1424,1024,1024,1024,400)")
    ap.add_argument("--batch-size", type=int, default=1024, help="training batch of --mlp")
    ap.add_argument("--basis", default="fp32", choices=sorted(_PREC))
    ap.add_argument("--recon", default="fp32", choices=sorted(_PREC))
    ap.add_argument("--taps", default="auto", choices=sorted(_TAPS), help="the residual's tap staging")
    ap.add_argument("--tuning", default=None, help="rows,row_chunks,col_groups,col_split (default: the "
                    "object's own geometry)")
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--profile-graph", action="store_true")
    ap.add_argument("--batch", type=int, default=0, help="this many realisations as one batch (shared DM and "
                    "bf16 reconstructor objects)")
    ap.add_argument("--persistent", action="store_true", help="the batch with PAS_BATCH_PERSISTENT")
    ap.add_argument("--seed", type=int, default=1)
    a = ap.parse_args(argv)
    if a.gemm > 0:
        return _gemm(a.gemm, a.steps, a.seed)
    if a.psf:
        return _psf(a.psf, a.steps, a.seed)
    if a.mlp:
        return _mlp(a.mlp, a.batch_size, a.steps, a.seed)
    cfg = get_config(a.workload)
    tuning = tuple(int(x) for x in a.tuning.split(",")) if a.tuning else False
    systems, loops, batch = [], [], None
    try:
        if a.batch > 0:
            first = _random_system(cfg, _PREC[a.basis], pas.PAS_BF16, tuning, a.seed)
            systems.append(first)
            for i in range(1, a.batch):
                systems.append(_random_system(with_(cfg, seed=cfg.seed + 17 * i), _PREC[a.basis], pas.PAS_BF16,
                                              tuning, a.seed, dm=first.dm, rec=first.rec, basis=first.basis,
                                              R=first.R))
        else:
            systems.append(_random_system(cfg, _PREC[a.basis], _PREC[a.recon], tuning, a.seed))
        for s in systems:
            pas.pas_atmo_set_tap_staging(s.atmo, s.ctx, _TAPS[a.taps])
            loops.append(pas.pas_loop_create(s.ctx, s.atmo, s.pyr, s.rec, s.dm, s.d_gain, s.delay, 64))
        ctx = systems[0].ctx
        if a.batch > 0:
            batch = pas.pas_batch_create_ex(ctx, loops, pas.PAS_BATCH_PERSISTENT if a.persistent else 0)
            pas.pas_batch_step(batch, ctx, a.steps)
            torch.cuda.synchronize()
            pas.pas_batch_check(batch, ctx)
        else:
            pas.pas_loop_step(loops[0], ctx, a.steps)
            if a.profile_graph:
                for _ in range(a.steps):
                    pas.pas_loop_profile(loops[0], ctx, 1)
        torch.cuda.synchronize()
        st, wfe = pas.pas_loop_step(loops[0], systems[0].ctx, 0, stats=True)
        print(f"{a.workload}: {st} steps, last residual WFE {wfe:.1f} nm (random system)")
        return 0
    finally:
        if batch is not None:
            pas.pas_batch_destroy(batch)
        for loop in loops:
            pas.pas_loop_destroy(loop)
        for s in systems[1:] + systems[:1]:
            s.close()


if __name__ == "__main__":
    raise SystemExit(main())
