#!/usr/bin/env python3
"""Benchmark: AO loop steps/s and PWFS frames/s on one GB300 (per rank).

Headline workload: the ELT-scale single-conjugate loop (39 m, 480 px pupil, 960^2
FFT grid, 6 layers, 96x96 pyramid, 32 modulation points at 4 lambda/D, 4000 modes,
noiseless), FP32. A step is one simulated millisecond: atmosphere + DM residual ->
modulated pyramid -> slopes -> reconstructor -> integrator, replayed as one CUDA
graph. The same loop with a bfloat16 DM basis and reconstructor, and the LBT-class
loop (240 px, 3 layers, photon and read noise), are reported beside it.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on
the launching stream, the L2 flushed (256 MiB write + read) between steps outside
the events; barrier + synchronize around the timed region, max over ranks.
Multi-GPU (torchrun): independent replicas (different seeds), weak scaling.

--impl reference times the FP64 CPU oracle on this machine's host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AO loop steps/s ({workload}, 1 GB300)"
UNIT = "steps/s"
FP32_PEAK_TFLOPS = None   # measured by the FMA probe at start-up (measure_fp32_peak)
FP32_PEAK_SOURCE = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="scao_elt_480px",
                    help="workload: scao_8m_64px, scao_lbt_240px or scao_elt_480px")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--recon", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--no-mlp", action="store_true", help="skip the learned-reconstructor measurements")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the BF16 loop and the other workloads (64 px, ELT-scale)")
    ap.add_argument("--soak", type=float, default=1.5, help="seconds of untimed steps before timing")
    ap.add_argument("--tuning", default=None,
                    help="pyramid launch geometry rows_per_cta,row_chunks,col_groups[,col_split] "
                         "(default: autotuned)")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-budget-s", type=float, default=20.0)
    ap.add_argument("--no-cpu-pool", action="store_true", help="skip the all-cores oracle timing")
    return ap.parse_args()


# ------------------------------------------------------------------ CPU oracle

def oracle_sample(workload: str, budget_s: float, max_steps: int) -> dict:
    """Time the FP64 oracle's closed-loop step (as it stands) for a bounded number
    of steps. Setup (screens, basis) is untimed; R is a seeded random matrix of
    the right shape (the timing does not depend on its values)."""
    import numpy as np
    from oracle import atmosphere as at
    from oracle import control as ct
    from oracle import modal as md
    from oracle import noise as nz
    from oracle import optics as op
    from synth import get_config
    from synth.inputs import layer_seeds, random_matrix, screen_white_noise
    cfg = get_config(workload)
    screens = at.layer_screens_nm(cfg, [screen_white_noise(cfg.S, s) for s in layer_seeds(cfg.seed, len(cfg.layers))])
    if cfg.n_modes > 1000:
        # a seeded random basis of the workload's shape: the step's cost does not
        # depend on its values (an orthonormal 4000-mode basis is a long setup)
        M = random_matrix(int(op.pupil_mask(cfg.Np, cfg.obs).sum()), cfg.n_modes, 4, 1.0)
    else:
        M = md.modal_basis(cfg.Np, cfg.obs, cfg.n_modes)
    valid = op.valid_subapertures(cfg.Np, cfg.obs, cfg.n_sub)
    R = random_matrix(cfg.n_modes, 2 * valid.size, 5, 1e-3)
    sn = np.zeros(2 * valid.size)
    noise = None
    if cfg.magnitude is not None:
        npup = int(op.pupil_mask(cfg.Np, cfg.obs).sum())
        noise = lambda fr, t: nz.apply_noise(fr, nz.photons_per_frame(cfg), npup, cfg.read_noise_e, cfg.seed, t)
    # one step to size the sample
    t0 = time.perf_counter()
    ct.closed_loop(cfg, screens, M, R, sn, valid, 1, noise=noise)
    t1 = time.perf_counter() - t0
    n = int(max(1, min(max_steps, budget_s // max(t1, 1e-6))))
    t0 = time.perf_counter()
    ct.closed_loop(cfg, screens, M, R, sn, valid, n, noise=noise)
    dt = time.perf_counter() - t0
    basis = "random basis" if cfg.n_modes > 1000 else "the oracle's basis"
    return {"steps": n, "seconds": dt, "value": n / dt,
            "sample": f"{n} closed-loop steps of {cfg.name} after one sizing step, FP64 NumPy oracle, 1 thread, "
                      f"{dt:.1f} s (setup untimed: screens, {basis}, random R of the right shape)"}


def run_oracle_subprocess(workload: str, budget_s: float, max_steps: int) -> dict:
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    with tempfile.NamedTemporaryFile("r", suffix=".json") as f:
        cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(max_steps), "--config",
               workload, "--oracle-budget-s", str(budget_s)]
        subprocess.run(cmd, env=env, check=True, stdout=open(f.name, "w"))
        return json.loads(open(f.name).read().strip().splitlines()[-1])


def run_oracle_pool(workload: str, budget_s: float, max_steps: int, n_proc: int) -> dict:
    """All host cores: n_proc independent copies of the oracle's closed loop (the
    oracle as it stands, one thread each), started together as fresh processes; the
    aggregate steps/s is the sum of their rates over their concurrent timed regions."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    outs, procs = [], []
    try:
        for _ in range(n_proc):
            f = tempfile.NamedTemporaryFile("r", suffix=".json")
            outs.append(f)
            cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(max_steps), "--config",
                   workload, "--oracle-budget-s", str(budget_s)]
            procs.append(subprocess.Popen(cmd, env=env, stdout=open(f.name, "w"), stderr=subprocess.DEVNULL))
        rates, steps = [], 0
        for p, f in zip(procs, outs):
            if p.wait() != 0:
                raise RuntimeError("an oracle process failed")
            r = json.loads(open(f.name).read().strip().splitlines()[-1])
            rates.append(r["value"])
            steps += r["steps"]
        return {"value": float(sum(rates)), "steps": steps, "processes": n_proc}
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
        for f in outs:
            f.close()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.path = tempfile.mktemp(suffix=".csv")
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nme, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nme)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ roofline

def algorithmic_work(cfg, n_pix, n_valid, n_modes, n_s_rows, recon_bytes_per_el, basis_bytes_per_el=4.0):
    """Per-launch algorithmic flops / bytes of each kernel of the step. An FFT of
    length N counts 5 N log2 N flops, the mask, tilt and |.|^2 work 6 N + 6 Np (+3 N
    in the columns pass for the binning and the modulation sum)."""
    N, Np, K, L = cfg.N, cfg.Np, cfg.K, len(cfg.layers)
    fft_pair = 2 * 5.0 * N * math.log2(N) + 6.0 * N           # FFT + mask + IFFT
    return {
        # basis block, pixel list and output, command, the layers' pupil footprints
        "residual_kernel": {"bound": "hbm", "bytes": basis_bytes_per_el * n_modes * n_pix + 8.0 * n_pix
                            + 4.0 * n_modes + 4.0 * L * (Np + 1) ** 2},
        "pyr_rows_kernel": {"bound": "alu", "flops": n_s_rows * Np * (fft_pair + 6.0 * Np)},
        "pyr_cols_kernel": {"bound": "alu", "flops": K * N * (fft_pair + 6.0 * Np + 3.0 * N)},
        "slopes_kernel": {"bound": "latency", "bytes": 16.0 * n_valid + 8.0 * 2 * n_valid},
        "recon_kernel": {"bound": "hbm", "bytes": recon_bytes_per_el * n_modes * 2 * n_valid + 8.0 * n_modes},
    }


def replica_seed(seed: int, rank: int) -> int:
    """Each replica simulates its own atmosphere (weak scaling, no data exchange)."""
    return seed + 1000 * rank


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's value (the job ends when every replica has finished)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job steps/s: the steps of all replicas over the slowest rank's time."""
    return steps_per_rank * world / (ms_max / 1000.0)


def timed_loop(sysg, timed, n_steps, warmup=20):
    """Reset the loop, warm it, reset again, time n_steps single-step graph launches
    (L2 flushed between steps by `timed`); returns (steps/s, per-step WFE)."""
    import numpy as np
    zeros = np.zeros((sysg.delay, sysg.n_modes), dtype=np.float32)
    sysg.set_state(0, zeros)
    sysg.step(warmup)
    sysg.set_state(0, zeros)
    ms = timed(lambda: sysg.step(1), n_steps)
    return n_steps / (ms * 1e-3), sysg.wfe_nm(min(n_steps, sysg.wfe_history))


def bench_bf16_loop(cfg_r, timed, n_steps, wfe_fp32):
    """The same loop (same seeds) with the DM basis and the reconstructor in bfloat16
    (float32 sums and integrator): steps/s and the residual WFE against the FP32 loop."""
    import numpy as np
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    sysb = SCAOSystem(cfg_r, recon_precision=pas.PAS_BF16, dm_precision=pas.PAS_BF16,
                      wfe_history=max(4096, n_steps + 64))
    try:
        sps, wfe = timed_loop(sysb, timed, n_steps)
    finally:
        sysb.close()
    n = min(len(wfe), len(wfe_fp32))
    burn = n // 5
    d = wfe[burn:n] - wfe_fp32[burn:n]
    d10 = wfe[:min(10, n)] - wfe_fp32[:min(10, n)]
    return {"steps_per_s": sps, "dm_basis": "bf16", "reconstructor": "bf16 (per-row scale)",
            "wfe_diff_nm_rms_first_10_steps": float(np.sqrt(np.mean(d10 * d10))),
            "wfe_nm_mean": float(np.mean(wfe[burn:n])), "wfe_nm_mean_fp32": float(np.mean(wfe_fp32[burn:n])),
            "wfe_diff_nm_rms": float(np.sqrt(np.mean(d * d))), "wfe_diff_nm_max": float(np.max(np.abs(d))),
            "steps_compared": n - burn}


def bench_other_workloads(timed, peaks, n_steps=200):
    """Loop steps/s and PWFS frames/s of the 64 px workload (Zernike basis,
    calibrated by push-pull on the GPU)."""
    import numpy as np
    import torch
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    from synth import get_config
    out = {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    cfg1 = get_config("scao_8m_64px")
    s1 = SCAOSystem(cfg1, wfe_history=max(4096, n_steps + 64))
    try:
        sps, _ = timed_loop(s1, timed, n_steps)
        opd = torch.zeros(cfg1.Np, cfg1.Np, device="cuda")
        pas.pas_atmo_advance(s1.atmo, s1.ctx, 0, opd)
        fr = n_steps / (timed(lambda: s1.measure(opd), n_steps) * 1e-3)
        out[cfg1.name] = {"loop_steps_per_s": sps, "pwfs_frames_per_s": fr, "tuning": list(s1.tuning)}
    finally:
        s1.close()
    return out


def bench_lbt(args, timed, barrier, flush, world, dist, peaks, no_mlp=False):
    """The LBT-class loop (8.4 m, 240 px, 3 layers, 400 KL modes calibrated on the
    GPU, magnitude-10 photon noise + 0.5 e- read noise), FP32: steps/s, PWFS
    frames/s, per-kernel rooflines and e2e as for the headline; the BF16 loop's WFE
    against it; the PSF camera attached to it; the learned reconstructor on its
    sizes. Returns (loop dict, learned-reconstructor dict or None)."""
    import numpy as np
    from paper_1607_07624_gb300 import pas
    from synth import get_config
    cfg = get_config("scao_lbt_240px")
    hist = max(4096, args.steps + args.warmup + 64)
    s = make_system(cfg, pas.PAS_FP32, pas.PAS_FP32, True, hist)
    mlp_info = None
    try:
        r = measure_loop(s, cfg, args, timed, barrier, flush, world, dist, peaks)
        wfe = r.pop("wfe")
        r["residual_wfe_nm_mean"] = float(np.mean(wfe[len(wfe) // 5:])) if len(wfe) else None
        r["tuning"] = list(s.tuning)
        r["inputs"] = s.setup_note
        try:
            r["loop_bf16"] = bench_bf16_loop(cfg, timed, args.steps, wfe)
        except Exception as e:
            r["loop_bf16"] = {"error": str(e)}
        try:
            r["psf_camera"] = bench_psf(timed, s)
        except Exception as e:
            r["psf_camera"] = {"error": str(e)}
        if not no_mlp:
            try:
                mlp_info = bench_mlp(s, peaks, timed)
            except Exception as e:  # reported, never fatal for the headline number
                mlp_info = {"error": str(e)}
    finally:
        s.close()
    return r, mlp_info


def bench_equal_wfe(timed, n_timed=300, workload="scao_lbt_240px", n_modes=200):
    """BF16 against FP32 at equal residual WFE where the loop settles: by default the LBT-class optics
    (240 px, 3 layers, magnitude-10 noise) with 200 KL modes (with 400 the linear loop
    drifts); also the ELT-scale optics (480 px, 6 layers, noiseless) with 1000 modes
    (with 4000 it drifts). The FP32 loop and the loop with a bfloat16 DM basis and
    reconstructor run the workload's steps from the same start; reported: their steps/s
    (L2 flushed between timed steps) and mean residual WFE after a 20 % burn-in."""
    import numpy as np
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    from synth import get_config
    from synth.configs import with_
    cfg = with_(get_config(workload), n_modes=n_modes)
    n = cfg.n_steps
    noise = f"magnitude {cfg.magnitude} noise" if cfg.magnitude is not None else "noiseless"
    out = {"workload": f"{cfg.name} with {cfg.n_modes} {cfg.basis} modes, {n} steps, {noise}"}
    a = SCAOSystem(cfg, wfe_history=n)
    try:
        b = SCAOSystem(cfg, basis=a.basis, R=a.R, recon_precision=pas.PAS_BF16, dm_precision=pas.PAS_BF16,
                       wfe_history=n, autotune=tuple(a.tuning))
        try:
            res = {}
            for label, s in (("fp32", a), ("bf16", b)):
                zeros = np.zeros((s.delay, s.n_modes), np.float32)
                s.set_state(0, zeros)
                s.step(n)
                w = s.wfe_nm(n)
                s.set_state(0, zeros)
                sps = n_timed / (timed(lambda: s.step(1), n_timed) * 1e-3)
                res[label] = {"steps_per_s": sps, "wfe_nm_mean": float(w[n // 5:].mean()),
                              "wfe_nm_first_step": float(w[0]), "wfe_nm_last_500_mean": float(w[-500:].mean())}
            out.update(res)
            out["wfe_diff_nm"] = res["bf16"]["wfe_nm_mean"] - res["fp32"]["wfe_nm_mean"]
            out["bf16_speedup"] = res["bf16"]["steps_per_s"] / res["fp32"]["steps_per_s"]
        finally:
            b.close()
    finally:
        a.close()
    return out


def cpu_baseline_for(cfg, args):
    """The FP64 oracle on this host: one thread, and all cores as independent
    single-thread loops (capped by host memory for the large workloads)."""
    try:
        r = run_oracle_subprocess(cfg.name, args.oracle_budget_s, 50)
        cpu = {"value": r["value"], "unit": UNIT, "cores": 1, "kind": "oracle", "sample": r["sample"]}
    except Exception as e:  # the baseline is reported, never fatal
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}
    if args.no_cpu_pool:
        return cpu
    n_proc = max(1, min(os.cpu_count() or 1, 16))
    try:
        phys = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        phys = None
    # an ELT-scale oracle process holds a 179 156 x 4000 FP64 basis (5.7 GB) and its copies
    per_proc = 16e9 if cfg.n_modes > 1000 else 2e9
    if phys:
        n_proc = max(1, min(n_proc, int(0.5 * phys // per_proc)))
    try:
        rp = run_oracle_pool(cfg.name, args.oracle_budget_s / 2, 50, n_proc)
        cpu["all_cores"] = {"value": rp["value"], "unit": UNIT, "cores": n_proc, "kind": "oracle",
                            "sample": f"{n_proc} independent closed loops of {cfg.name} in {n_proc} "
                                      f"single-thread processes started together, {rp['steps']} steps "
                                      f"in all (steps/s summed over the concurrent loops)"}
    except Exception as e:
        cpu["all_cores"] = {"value": None, "cores": n_proc, "sample": f"failed: {e}"}
    return cpu


def bench_psf(timed, sysg=None, n_frames=100):
    """PSF camera on the LBT-class optics at the paper's camera settings (1650 nm,
    padding 8: a 1920 x 1920 grid), integrating every frame into a long-exposure PSF:
    frames/s and the FP32 roofline of its two FFT passes. The residual is a smooth
    closed-loop-like OPD of 150 nm RMS."""
    import numpy as np
    import torch
    from paper_1607_07624_gb300 import pas
    from synth import get_config
    from synth.inputs import random_opd_nm
    cfg = get_config("scao_lbt_240px")
    Np, nd = cfg.Np, 8
    ctx = pas.pas_ctx_create(torch.cuda.current_stream())
    h = pas.pas_psf_create(ctx, Np, nd, 1650.0, cfg.obs)
    try:
        N = pas.pas_psf_size(h)
        opd = torch.as_tensor(random_opd_nm(Np, 150.0, seed=3).astype(np.float32)).cuda()
        acc = torch.zeros(N, N, device="cuda")
        sr = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(5):
            pas.pas_psf_compute(h, ctx, opd, acc, True, sr)
        ms = timed(lambda: pas.pas_psf_compute(h, ctx, opd, acc, True, sr), n_frames)
        torch.cuda.synchronize()
        per = ms / n_frames * 1e-3
        # FFTs of the Np pupil columns and the N frequency rows, |.|^2 and the sum
        flops = (Np + N) * 5.0 * N * math.log2(N) + 4.0 * N * N
        bytes_ = 8.0 * N * N + 4.0 * Np * Np + 2 * 8.0 * N * Np   # PSF read+write, OPD, intermediate
        ach = flops / per / 1e12
        out = {"workload": f"PSF {N}x{N} (Np {Np}, nd {nd}, 1650 nm), integrated each frame",
               "frames_per_s": n_frames / (ms * 1e-3), "us_per_frame": per * 1e6,
               "strehl": float(sr.item()), "flops_per_frame": flops, "bytes_per_frame": bytes_,
               "roofline": {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": ach / FP32_PEAK_TFLOPS}}
        if sysg is not None:
            # the LBT-class loop with the camera integrating every step (the camera's two
            # kernels on a branch of the loop's step graph), then the loop state is restored
            zeros = np.zeros((sysg.delay, sysg.n_modes), dtype=np.float32)
            sysg.attach_camera(nd=nd, wavelength_nm=1650.0, start_step=0)
            try:
                sysg.set_state(0, zeros)
                sysg.step(5)
                sysg.set_state(0, zeros)
                ms_l = timed(lambda: sysg.step(1), n_frames)
                torch.cuda.synchronize()
                out["loop_with_camera_steps_per_s"] = n_frames / (ms_l * 1e-3)
                out["loop_with_camera_mean_strehl"] = float(sysg.sr[:n_frames].mean().item())
            finally:
                sysg.detach_camera()
                sysg.set_state(0, zeros)
        return out
    finally:
        pas.pas_psf_destroy(h)
        pas.pas_ctx_destroy(ctx)


def bench_sh(timed, n_frames=200):
    """Shack-Hartmann sensor on the LBT-class geometry (240 px pupil, 30 x 30 lenslets of
    8 px, Nyquist spots of 16 x 16 px, 750 nm): frame + slopes per measurement,
    frames/s, and the FP32 roofline of the lenslet DFTs (two dense products per
    lenslet: b M b + M M b complex multiply-adds)."""
    import numpy as np
    import torch
    from paper_1607_07624_gb300 import pas
    from synth import get_config
    from synth.inputs import random_opd_nm
    cfg = get_config("scao_lbt_240px")
    Np, n_sub, ovs = cfg.Np, cfg.n_sub, 2
    ctx = pas.pas_ctx_create(torch.cuda.current_stream())
    h = pas.pas_sh_create(ctx, Np, n_sub, ovs, cfg.wavelength_nm, cfg.obs)
    try:
        side, nv = pas.pas_sh_frame_side(h), pas.pas_sh_n_valid(h)
        opd = torch.as_tensor(random_opd_nm(Np, 150.0, seed=3).astype(np.float32)).cuda()
        fr = torch.zeros(side, side, device="cuda")
        sl = torch.zeros(2 * nv, device="cuda")
        for _ in range(5):
            pas.pas_sh_measure(h, ctx, opd, fr, sl)
        ms = timed(lambda: pas.pas_sh_measure(h, ctx, opd, fr, sl), n_frames)
        torch.cuda.synchronize()
        b = Np // n_sub
        M = ovs * b
        flops = n_sub * n_sub * 8.0 * (b * M * b + M * M * b)
        per = ms / n_frames * 1e-3
        ach = flops / per / 1e12
        out = {"workload": f"Shack-Hartmann {n_sub}x{n_sub} lenslets of {b} px, {M}x{M} spots, {nv} valid",
               "frames_per_s": n_frames / (ms * 1e-3), "us_per_frame": per * 1e6, "flops_per_frame": flops,
               "roofline": {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": ach / FP32_PEAK_TFLOPS}}
    finally:
        pas.pas_sh_destroy(h)
        pas.pas_ctx_destroy(ctx)
    # the closed loop with this sensor in place of the pyramid (noiseless; same
    # atmosphere, KL basis and integrator; calibrated by push-pull through the sensor)
    from paper_1607_07624_gb300.system import SCAOSystem
    s = SCAOSystem(cfg, sensor="sh", sh_ovs=ovs, wfe_history=max(4096, n_frames + 64))
    try:
        sps, wfe = timed_loop(s, timed, n_frames)
        out["loop_steps_per_s"] = sps
        out["loop_wfe_nm_first_steps"] = [float(x) for x in wfe[:5]]
    finally:
        s.close()
    return out


def bench_extended(timed, n_frames=100):
    """The LBT-class pyramid looking at an extended source, a 3 x 3 grid of points over
    2 lambda/D (K x 9 = 216 tilt points, 13 x 3 = 39 rows passes): frames/s, the FP32
    roofline of its transforms (rows passes plus the 216 column transforms, the
    point-source formulas with K x 9 points) and the closed loop with this sensor."""
    import numpy as np
    import torch
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    from synth import get_config
    from synth.configs import with_
    cfg = get_config("scao_lbt_240px")
    g = np.linspace(-1.0, 1.0, 3)
    ex, ey = np.repeat(g, 3), np.tile(g, 3)
    s = SCAOSystem(cfg, extended_source=(ex, ey), wfe_history=max(4096, n_frames + 64))
    try:
        opd = torch.zeros(cfg.Np, cfg.Np, dtype=torch.float32, device="cuda")
        pas.pas_atmo_advance(s.atmo, s.ctx, 0, opd)
        for _ in range(3):
            s.measure(opd)
        ms = timed(lambda: s.measure(opd), n_frames)
        n_rows = (cfg.K // 2 + 1 if cfg.K % 2 == 0 else cfg.K) * len(set(ey.tolist()))
        work = algorithmic_work(with_(cfg, K=cfg.K * ex.size), s.n_pix, s.n_valid, s.n_modes, n_rows, 4.0)
        flops = work["pyr_rows_kernel"]["flops"] + work["pyr_cols_kernel"]["flops"]
        per = ms / n_frames * 1e-3
        ach = flops / per / 1e12
        out = {"workload": f"pyramid {cfg.Np} px, K {cfg.K}, extended source of {ex.size} points over 2 lambda/D",
               "frames_per_s": n_frames / (ms * 1e-3), "us_per_frame": per * 1e6, "flops_per_frame": flops,
               "tilt_points": cfg.K * ex.size, "rows_passes": n_rows, "tuning": list(s.tuning),
               "roofline": {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": ach / FP32_PEAK_TFLOPS}}
        sps, wfe = timed_loop(s, timed, n_frames)
        out["loop_steps_per_s"] = sps
        out["loop_wfe_nm_first_steps"] = [float(x) for x in wfe[:5]]
        return out
    finally:
        s.close()


def bench_batch(timed, n_loops=64, n_steps=100):
    """Monte-Carlo batch: n_loops realisations of the 64 px workload (own screens
    each; DM object, reconstructor matrix and launch geometry shared, so the batch
    computes their residuals in one basis pass) stepped by one graph launch per step,
    as graph branches and with the persistent pyramid launch. Returns the whole batch's
    loop-steps/s for the faster, both modes beside it. Also the batched BF16 loop: the
    same realisations sharing one bf16 reconstructor object (one tensor-core product per
    step for all of them), its rate and its residual WFE against the FP32 batch's."""
    import numpy as np
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    from synth import get_config
    from synth.configs import with_
    cfg = get_config("scao_8m_64px")
    systems = [SCAOSystem(cfg, wfe_history=max(256, n_steps + 64))]
    batch = None
    try:
        for i in range(1, n_loops):
            systems.append(SCAOSystem(with_(cfg, seed=cfg.seed + 7919 * i), basis=systems[0].basis, R=systems[0].R,
                                      dm=systems[0].dm, autotune=tuple(systems[0].tuning),
                                      wfe_history=max(256, n_steps + 64)))
        modes, wfe = {}, None
        for name, flags in (("graph_branches", 0), ("persistent", pas.PAS_BATCH_PERSISTENT)):
            batch = pas.pas_batch_create_ex(systems[0].ctx, [s.loop for s in systems], flags)
            pas.pas_batch_step(batch, systems[0].ctx, 5)
            for s in systems:
                s.set_state(0, np.zeros((s.delay, s.n_modes), np.float32))
            ms = timed(lambda: pas.pas_batch_step(batch, systems[0].ctx, 1), n_steps)
            pas.pas_batch_check(batch, systems[0].ctx)
            modes[name] = {"loop_steps_per_s": n_loops * n_steps / (ms * 1e-3),
                           "batch_steps_per_s": n_steps / (ms * 1e-3),
                           "kernels_per_step": pas.pas_batch_kernels_per_step(batch)}
            if wfe is None:
                wfe = np.array([s.wfe_nm(n_steps) for s in systems])
            pas.pas_batch_destroy(batch)
            batch = None
        best = max(modes, key=lambda k: modes[k]["loop_steps_per_s"])
        out = {"workload": f"{n_loops} realisations of {cfg.name} (own screens each)", "mode": best, **modes[best],
               "graph_launches_per_step": 1, "modes": modes,
               "wfe_nm_mean_over_realisations": float(wfe[:, n_steps // 5:].mean())}
        out["bf16_shared_reconstructor"] = _bench_batch_bf16(timed, cfg, systems, n_steps, wfe)
        return out
    finally:
        if batch is not None:
            pas.pas_batch_destroy(batch)
        for s in systems[1:] + systems[:1]:
            s.close()


def _bench_batch_bf16(timed, cfg, systems, n_steps, wfe_fp32):
    """The Monte-Carlo batch's realisations again (same seeds, basis, DM object) with one
    shared bf16 reconstructor object: graph branches plus one tensor-core product per
    step. Reports loop-steps/s and the WFE against the FP32 batch (mean after a 20 %
    burn-in, over realisations, and the largest per-realisation difference)."""
    import numpy as np
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    from synth.configs import with_
    first = systems[0]
    rec = pas.pas_recon_create(first.ctx, first.R, pas.PAS_BF16)
    twins, batch = [], None
    try:
        for i, s in enumerate(systems):
            twins.append(SCAOSystem(with_(cfg, seed=cfg.seed + 7919 * i) if i else cfg, basis=first.basis, R=first.R,
                                    dm=first.dm, rec=rec, autotune=tuple(first.tuning), wfe_history=s.wfe_history))
        batch = pas.pas_batch_create(first.ctx, [t.loop for t in twins])
        pas.pas_batch_step(batch, first.ctx, 5)
        for t in twins:
            t.set_state(0, np.zeros((t.delay, t.n_modes), np.float32))
        ms = timed(lambda: pas.pas_batch_step(batch, first.ctx, 1), n_steps)
        pas.pas_batch_check(batch, first.ctx)
        w = np.array([t.wfe_nm(n_steps) for t in twins])
        b0 = n_steps // 5
        per = w[:, b0:].mean(axis=1) - wfe_fp32[:, b0:].mean(axis=1)
        return {"loop_steps_per_s": len(twins) * n_steps / (ms * 1e-3),
                "kernels_per_step": pas.pas_batch_kernels_per_step(batch),
                "tensor_core_reconstruction_groups": pas.pas_batch_n_groups(batch),
                "wfe_nm_mean_bf16": float(w[:, b0:].mean()), "wfe_nm_mean_fp32": float(wfe_fp32[:, b0:].mean()),
                "wfe_diff_nm_max_over_realisations": float(np.abs(per).max())}
    finally:
        if batch is not None:
            pas.pas_batch_destroy(batch)
        for t in twins:
            t.close()
        pas.pas_recon_destroy(rec)


def bench_batched_workload(timed, n_steps=30):
    """The batched Monte-Carlo workload: 64 loops of three sizes (32 x 128 px with
    20x20 sub-apertures, 24 x 320 px with 60x60, 8 x 480 px with 96x96; 6.4, 5.33
    and 5 pixels per sub-aperture), each with its own screens (seed and r0 drawn
    in 0.08-0.2 m), stepped by one graph launch per step. The loops of a group are
    realisations of one system: they share one DM object (a random basis of the
    group's shape) and one bf16 reconstructor object (random, of its shape), so the
    batch reconstructs each group with one tensor-core product; the pyramid launch
    geometry is autotuned once per group: timing only, the wavefront error is not
    meaningful."""
    import numpy as np
    import torch
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    from synth.configs import batched_workload
    gen = torch.Generator(device="cuda").manual_seed(11)
    ctx = pas.pas_ctx_create(torch.cuda.current_stream())
    systems, shared, batch = [], {}, None
    try:
        for gi, cfg in batched_workload():
            if gi not in shared:
                pix = pas.pas_pupil_pixels(cfg.Np, cfg.obs)
                valid = pas.pas_valid_subaps(cfg.Np, cfg.obs, cfg.n_sub)
                basis = torch.randn(pix.size, cfg.n_modes, device="cuda", generator=gen).cpu().numpy()
                R = (torch.randn(cfg.n_modes, 2 * valid.size, device="cuda", generator=gen) * 1e-3).cpu().numpy()
                shared[gi] = {"basis": basis, "R": R, "dm": pas.pas_dm_create(ctx, basis, cfg.Np, cfg.obs),
                              "rec": pas.pas_recon_create(ctx, np.ascontiguousarray(R, dtype=np.float32),
                                                          pas.PAS_BF16),
                              "tuning": True, "name": cfg.name, "count": 0, "n_valid": int(valid.size),
                              "n_modes": cfg.n_modes}
            sh = shared[gi]
            sysl = SCAOSystem(cfg, basis=sh["basis"], R=sh["R"], dm=sh["dm"], rec=sh["rec"],
                              autotune=sh["tuning"], wfe_history=max(256, n_steps + 64))
            if sh["tuning"] is True:
                sh["tuning"] = tuple(sysl.tuning)
            sh["count"] += 1
            systems.append(sysl)
        modes = {}
        for name, flags in (("graph_branches", 0), ("persistent", pas.PAS_BATCH_PERSISTENT)):
            batch = pas.pas_batch_create_ex(ctx, [s.loop for s in systems], flags)
            pas.pas_batch_step(batch, ctx, 3)
            for s in systems:
                s.set_state(0, np.zeros((s.delay, s.n_modes), np.float32))
            ms = timed(lambda: pas.pas_batch_step(batch, ctx, 1), n_steps)
            pas.pas_batch_check(batch, ctx)
            modes[name] = {"ms_per_batch_step": ms / n_steps,
                           "loop_steps_per_s": len(systems) * n_steps / (ms * 1e-3),
                           "kernels_per_step": pas.pas_batch_kernels_per_step(batch),
                           "persistent_launches_per_step": pas.pas_batch_n_persistent(batch),
                           "tensor_core_reconstruction_groups": pas.pas_batch_n_groups(batch),
                           "shared_dm_residual_groups": pas.pas_batch_n_residual_groups(batch)}
            if flags:
                modes[name]["persistent_geometry"] = [pas.pas_batch_persistent_geometry(batch, ctx, g)
                                                      for g in range(pas.pas_batch_n_persistent(batch))]
            pas.pas_batch_destroy(batch)
            batch = None
        best = max(modes, key=lambda k: modes[k]["loop_steps_per_s"])
        groups = [{k: v for k, v in sh.items() if k in ("name", "count", "n_valid", "n_modes", "tuning")}
                  for sh in shared.values()]
        return {"loops": len(systems), "groups": groups, "mode": best, **modes[best],
                "graph_launches_per_step": 1, "modes": modes,
                "note": "random bases and reconstructors of the workload's shapes, shared within a group: "
                        "timing only"}
    finally:
        if batch is not None:
            pas.pas_batch_destroy(batch)
        for s in systems:
            s.close()
        torch.cuda.synchronize()
        for sh in shared.values():
            pas.pas_dm_destroy(sh["dm"])
            pas.pas_recon_destroy(sh["rec"])
        pas.pas_ctx_destroy(ctx)


def bench_mlp(sysg, peaks, timed, n_train=50, batch=1024):
    """Learned reconstructor on this system's sizes (2 n_valid -> 1024^3 -> n_modes):
    training throughput (Adam steps on a device-resident synthetic set larger than
    L2, one CUDA-graph replay per step, timed back to back), a large standalone
    tensor-core GEMM against the measured bf16 peak with cuBLAS beside it, and the
    loop with the network as its reconstructor."""
    import numpy as np
    import torch
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.learned import MLPReconstructor, he_normal_params
    ctx = sysg.ctx
    sizes = [2 * sysg.n_valid, 1024, 1024, 1024, sysg.n_modes]
    mlp = MLPReconstructor(ctx, sizes, max_batch=batch, seed=7)
    gen = torch.Generator(device="cuda").manual_seed(7)
    n_data = 65536
    S = torch.randn(n_data, sizes[0], device="cuda", generator=gen)
    Y = torch.randn(n_data, sizes[-1], device="cuda", generator=gen)
    idx = torch.randint(0, n_data, (n_train * batch,), device="cuda", generator=gen, dtype=torch.int32)
    lr = torch.full((n_train,), 1e-4, device="cuda")
    loss = torch.zeros(n_train, device="cuda")
    pas.pas_mlp_train(mlp.h, ctx, S, Y, n_data, batch, idx, lr, 5, loss)  # captures the step graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("train")
    e0.record()
    pas.pas_mlp_train(mlp.h, ctx, S, Y, n_data, batch, idx, lr, n_train, loss)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    pas.pas_mlp_check(mlp.h, ctx)
    ms = e0.elapsed_time(e1) / n_train
    mac = sum(a * b for a, b in zip(sizes[:-1], sizes[1:]))
    flops = 2.0 * batch * (2 * mac + (mac - sizes[0] * sizes[1]))  # forward, weight and input gradients
    bf16_sus = peaks.get("bf16_tflops_sustained", 1700.0)
    bf16_burst = peaks.get("bf16_tflops", 1900.0)
    train = {"batch": batch, "ms_per_step": ms, "samples_per_s": batch / (ms * 1e-3),
             "flops_per_step": flops, "tflops": flops / (ms * 1e-3) / 1e12,
             "frac_of_bf16_sustained": flops / (ms * 1e-3) / 1e12 / bf16_sus,
             "note": "whole Adam step (GEMMs + input, loss, bias-gradient and Adam kernels), one graph replay"}
    # the same step at batch 4096 (four times the GEMM work per step)
    mlp4 = MLPReconstructor(ctx, sizes, max_batch=4 * batch, seed=7)
    n4 = max(1, n_train // 4)
    idx4 = torch.randint(0, n_data, (n4 * 4 * batch,), device="cuda", generator=gen, dtype=torch.int32)
    pas.pas_mlp_train(mlp4.h, ctx, S, Y, n_data, 4 * batch, idx4, lr, 2, loss)
    torch.cuda.synchronize()
    e0.record()
    pas.pas_mlp_train(mlp4.h, ctx, S, Y, n_data, 4 * batch, idx4, lr, n4, loss)
    e1.record()
    torch.cuda.synchronize()
    pas.pas_mlp_check(mlp4.h, ctx)
    mlp4.close()
    ms4 = e0.elapsed_time(e1) / n4
    train["batch_4096"] = {"ms_per_step": ms4, "samples_per_s": 4 * batch / (ms4 * 1e-3),
                           "tflops": 4 * flops / (ms4 * 1e-3) / 1e12}
    del S, Y
    # standalone GEMM C = A B^T, 8192^3, operands 2 x 128 MiB (larger than L2), back to back
    n = 8192
    A = torch.randn(n, n, device="cuda", generator=gen).to(torch.bfloat16)
    B = torch.randn(n, n, device="cuda", generator=gen).to(torch.bfloat16)
    C = torch.empty(n, n, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(3):
        pas.pas_gemm_bf16(ctx, n, n, n, A, n, B, n, C, n, err)
    torch.cuda.synchronize()
    reps = 10
    torch.cuda.nvtx.range_push("gemm")
    e0.record()
    for _ in range(reps):
        pas.pas_gemm_bf16(ctx, n, n, n, A, n, B, n, C, n, err)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ours = 2.0 * n ** 3 / (e0.elapsed_time(e1) / reps * 1e-3) / 1e12
    for _ in range(3):
        torch.matmul(A, B.t())
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        torch.matmul(A, B.t())
    e1.record()
    torch.cuda.synchronize()
    cub = 2.0 * n ** 3 / (e0.elapsed_time(e1) / reps * 1e-3) / 1e12
    gemm = {"shape": [n, n, n], "tflops": ours, "peak": bf16_burst, "frac": ours / bf16_burst,
            "timeout_flag": int(err.item()), "cublas_bf16_tflops": cub,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (of measured, burst)"}
    del A, B, C
    # loop with the network (hidden layers He-initialised, output layer zero: same work, bounded state)
    p = he_normal_params(sizes, 7)
    p[-(sizes[-1] * sizes[-2] + sizes[-1]):] = 0.0
    mlp.set_params(p)
    pas.pas_loop_set_mlp(sysg.loop, ctx, mlp.h)
    sysg.set_state(0, np.zeros((sysg.delay, sysg.n_modes), dtype=np.float32))
    sysg.step(20)
    n_loop = 200
    torch.cuda.nvtx.range_push("timed_network")
    ms_loop = timed(lambda: sysg.step(1), n_loop)
    torch.cuda.nvtx.range_pop()
    chain = pas.pas_loop_profile(sysg.loop, ctx, 20).get("recon_kernel")
    try:
        batched = _bench_batched_network(sysg, mlp, timed)
    except Exception as e:  # reported, never fatal
        batched = {"error": str(e)}
    pas.pas_loop_set_mlp(sysg.loop, ctx, None)
    mlp.close()
    return {"sizes": sizes, "train": train, "gemm": gemm,
            "loop_steps_per_s_with_network": n_loop / (ms_loop * 1e-3),
            "network_chain_ms_in_loop": chain, "batched": batched}


def _bench_batched_network(sysg, mlp, timed, n_loops=8, n_steps=50):
    """n_loops realisations of this system (own screens; basis, R, DM object and launch
    geometry shared) stepped as one batch, one graph launch per step: all of them with one
    shared network (one batched tensor-core forward per step, bf16 activations) and, for
    comparison, all with the linear FP32 reconstructor. Loop-steps/s, L2 flushed between
    steps."""
    import numpy as np
    from paper_1607_07624_gb300 import pas
    from paper_1607_07624_gb300.system import SCAOSystem
    from synth.configs import with_
    cfg = sysg.cfg
    twins = []
    try:
        for i in range(1, n_loops):
            twins.append(SCAOSystem(with_(cfg, seed=cfg.seed + 7919 * i), basis=sysg.basis, R=sysg.R, dm=sysg.dm,
                                    autotune=tuple(sysg.tuning), wfe_history=256))
        members = [sysg] + twins
        out = {"loops": n_loops}
        for name in ("shared_network", "linear_fp32"):
            for s in members:
                pas.pas_loop_set_mlp(s.loop, s.ctx, mlp.h if name == "shared_network" else None)
            batch = pas.pas_batch_create(sysg.ctx, [s.loop for s in members])
            try:
                for s in members:
                    s.set_state(0, np.zeros((s.delay, s.n_modes), np.float32))
                pas.pas_batch_step(batch, sysg.ctx, 5)
                ms = timed(lambda: pas.pas_batch_step(batch, sysg.ctx, 1), n_steps)
                pas.pas_batch_check(batch, sysg.ctx)
                out[name] = {"loop_steps_per_s": n_loops * n_steps / (ms * 1e-3),
                             "kernels_per_step": pas.pas_batch_kernels_per_step(batch),
                             "batched_groups": pas.pas_batch_n_groups(batch)}
            finally:
                pas.pas_batch_destroy(batch)
        return out
    finally:
        for s in twins:
            pas.pas_loop_set_mlp(s.loop, s.ctx, None)
            s.close()


def measure_fp32_peak(stream, reps=20, iters=4096, blocks_per_sm=8):
    """FP32 FMA throughput of this GPU (pas_fp32_fma_probe over every SM, 2048 threads
    per SM, each with 8 independent FMA chains), timed with CUDA events on the
    launching stream: median and best of `reps` launches after a warm-up."""
    import torch
    from paper_1607_07624_gb300 import pas
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    n_blocks = sms * blocks_per_sm
    sink = torch.empty(n_blocks * 256, device="cuda")
    for _ in range(3):
        flops = pas.pas_fp32_fma_probe(sink, n_blocks, iters, stream)
    torch.cuda.synchronize()
    rates = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pas.pas_fp32_fma_probe(sink, n_blocks, iters, stream)
        b.record(stream)
        b.synchronize()
        rates.append(flops / (a.elapsed_time(b) * 1e-3) / 1e12)
    return {"tflops": statistics.median(rates), "tflops_best": max(rates), "sms": sms,
            "nominal_at_max_clock": sms * 128 * 2 * 2.070e9 / 1e12,
            "how": f"pas_fp32_fma_probe: {n_blocks} CTAs x 256 threads x 8 FMA chains x {iters} rounds, "
                   f"median of {reps} launches (CUDA events)"}


_SETUP_CACHE: dict = {}


def make_system(cfg, prec, dm_prec, tuning, wfe_history):
    """The workload's loop, calibrated: its modal basis (KL up to 1000 modes; above,
    the orthonormal Zernike basis of the same span, Cholesky QR on the GPU), the
    push-pull interaction matrix measured on the GPU and its FP64 Jacobi-SVD
    pseudo-inverse on the GPU. The basis and reconstructor are kept for the next
    system of the same workload (the BF16 variant)."""
    from paper_1607_07624_gb300.system import SCAOSystem
    kw = {k: v for k, v in _SETUP_CACHE.get(cfg.name, {}).items() if k in ("basis", "R")}
    sysg = SCAOSystem(cfg, recon_precision=prec, dm_precision=dm_prec, wfe_history=wfe_history, autotune=tuning,
                      **kw)
    if not kw:
        _SETUP_CACHE[cfg.name] = {"basis": sysg.basis, "R": sysg.R}
        sysg.setup_note = (f"von Karman screens; {sysg.n_modes}-mode basis: {sysg.basis_kind}; push-pull "
                           f"interaction matrix on the GPU, FP64 Jacobi-SVD pseudo-inverse on the GPU "
                           f"(rank {getattr(sysg, 'im_rank', None)}, {getattr(sysg, 'pinv_sweeps', None)} sweeps)")
        _SETUP_CACHE[cfg.name]["note"] = sysg.setup_note
    else:
        sysg.setup_note = _SETUP_CACHE[cfg.name]["note"]
    return sysg


def roofline_rows(cfg, sysg, prof, prec_bytes, peaks):
    n_s_rows = cfg.K // 2 + 1 if cfg.K % 2 == 0 else cfg.K
    work = algorithmic_work(cfg, sysg.n_pix, sysg.n_valid, sysg.n_modes, n_s_rows, prec_bytes,
                            basis_bytes_per_el=sysg.basis_bytes_per_el)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    roof = []
    for k, ms in prof.items():
        w = work.get(k)
        if not w or ms <= 0:
            continue
        if w["bound"] == "alu":
            ach = w["flops"] / (ms * 1e-3) / 1e12
            roof.append({"kernel": k, "ms": ms, "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS, "flops": w["flops"],
                         "peak_source": FP32_PEAK_SOURCE})
        else:
            ach = w["bytes"] / (ms * 1e-3) / 1e9
            roof.append({"kernel": k, "ms": ms, "bound": w["bound"], "achieved": ach, "peak": hbm_peak,
                         "unit": "GB/s", "frac": ach / hbm_peak, "bytes": w["bytes"],
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"})
    return roof


def measure_loop(sysg, cfg, args, timed, barrier, flush, world, dist, peaks, e2e=True):
    """Steps/s of the whole step graph, PWFS frames/s, per-kernel profile and rooflines,
    and the end-to-end rate through the public API with host copies."""
    import numpy as np
    import torch
    from paper_1607_07624_gb300 import pas
    stream = torch.cuda.current_stream()
    sysg.step(max(3, args.warmup))
    t_end = time.perf_counter() + args.soak
    while time.perf_counter() < t_end:
        sysg.step(50)
    barrier()
    sysg.set_state(0, np.zeros((sysg.delay, sysg.n_modes), dtype=np.float32))
    barrier()
    t_wall = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")
    ms_total = timed(lambda: sysg.step(1), args.steps)
    torch.cuda.nvtx.range_pop()
    barrier()
    t_wall = time.perf_counter() - t_wall
    ms_total = max_over_ranks(ms_total, dist, "cuda")
    out = {"value": job_throughput(args.steps, world, ms_total), "ms_per_step": ms_total / args.steps,
           "wall_timed_s": t_wall}
    # PWFS frames/s: the sensor alone on the open-loop OPD of step 0
    opd = torch.zeros(cfg.Np, cfg.Np, dtype=torch.float32, device="cuda")
    pas.pas_atmo_advance(sysg.atmo, sysg.ctx, 0, opd)
    n_fr = max(20, min(args.steps, 500))
    out["pwfs_frames_per_s"] = world * n_fr / (timed(lambda: sysg.measure(opd), n_fr) / 1000.0)
    # per-kernel durations (eager step with events around each kernel, L2 flushed)
    prof = {}
    n_prof = max(10, min(args.steps, 100))
    for _ in range(n_prof):
        flush.zero_()
        for k, v in pas.pas_loop_profile(sysg.loop, sysg.ctx, 1).items():
            prof[k] = prof.get(k, 0.0) + v / n_prof
    out["kernel_ms"] = prof
    out["roofline_by_kernel"] = roofline_rows(cfg, sysg, prof, sysg.recon_bytes_per_el, peaks)
    wfe = sysg.wfe_nm(min(sysg.wfe_history, args.steps))
    out["wfe"] = wfe
    if e2e:
        # end to end through the public API, host buffers: per step one graph launch
        # (pas_loop_step), then the new modal command and the step's residual WFE are
        # copied to pinned host memory and the stream is synchronised once
        n_e2e = max(20, min(args.steps, 300))
        cmd_host = torch.empty(sysg.n_modes, dtype=torch.float32, pin_memory=True)
        wfe_host = torch.empty(1, dtype=torch.float64, pin_memory=True)
        step0, _ = sysg.get_state()
        barrier()
        t0 = time.perf_counter()
        for i in range(n_e2e):
            sysg.step(1)
            cmd_host.copy_(sysg.loop_cmd, non_blocking=True)
            k = (step0 + i) % sysg.wfe_history
            wfe_host.copy_(sysg.loop_wfe[k:k + 1], non_blocking=True)
            stream.synchronize()
        e2e_s = time.perf_counter() - t0
        barrier()
        out["e2e"] = {"value": n_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                      "d2h_bytes_per_step": 4 * sysg.n_modes + 8,
                      "inputs": "device-resident loop state: the atmosphere's layers are uploaded once and "
                                "advanced on the GPU, so a step has no per-step input to copy; each step "
                                "copies its new modal command and residual WFE to pinned host memory and "
                                "synchronises once"}
    return out


def main():
    global FP32_PEAK_TFLOPS, FP32_PEAK_SOURCE
    args = parse()
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.config, args.oracle_budget_s, args.oracle_sample)))
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    from synth import get_config
    cfg = get_config(args.config)

    if args.impl == "reference":
        if rank != 0:
            return
        r = run_oracle_subprocess(args.config, args.oracle_budget_s, max(1, args.steps))
        line = {"impl": "reference", "metric": METRIC.format(workload=cfg.name), "value": r["value"], "unit": UNIT, "n_gpus": args.gpus,
                "steps": r["steps"], "warmup": 1, "ms_per_step": 1000.0 / r["value"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": cfg.name, "note": "FP64 NumPy oracle, single thread"},
                "cpu_baseline": {"kind": "oracle", "cores": 1, "value": r["value"], "unit": UNIT,
                                 "sample": r["sample"]},
                "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import numpy as np
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_1607_07624_gb300 import pas
    from synth.configs import with_

    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(local_rank)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler(f"GPU-{uuid}" if uuid else None) if rank == 0 else None
    fp32 = measure_fp32_peak(stream)
    FP32_PEAK_TFLOPS = fp32["tflops"]
    FP32_PEAK_SOURCE = f"measured: FP32 FMA probe on {fp32['sms']} SMs (median), this run"
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass

    cfg_r = with_(cfg, seed=replica_seed(cfg.seed, rank))
    prec = pas.PAS_BF16 if args.recon == "bf16" else pas.PAS_FP32
    tuning = tuple(int(v) for v in args.tuning.split(",")) if args.tuning else True
    hist = max(4096, args.steps + args.warmup + 64)
    t_setup = time.perf_counter()
    sysg = make_system(cfg_r, prec, pas.PAS_FP32, tuning, hist)
    t_setup = time.perf_counter() - t_setup
    # L2 flush between timed steps: write 256 MiB (evicts everything), then read
    # another 256 MiB so that the dirty lines are written back outside the timed
    # region and the next step starts from a clean, cold L2
    flush_w = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_sink = torch.zeros(1, dtype=torch.float32, device="cuda")

    class _Flush:
        @staticmethod
        def zero_():
            flush_w.zero_()
            torch.sum(flush_r, dim=0, keepdim=True, out=flush_sink)

    flush = _Flush()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, n):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    head = measure_loop(sysg, cfg, args, timed, barrier, flush, world, dist, peaks)
    roof = head["roofline_by_kernel"]
    dom = max(roof, key=lambda r: r["ms"]) if roof else None
    pwfs_roof = next((r for r in roof if r["kernel"] == "pyr_cols_kernel"), None)
    traffic = None
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        traffic = tr.get(cfg.name, {}).get(dom["kernel"]) if dom else None
    except (OSError, ValueError):
        pass
    setup_note = sysg.setup_note
    sysg.close()

    extra = {}
    mlp_info = None
    # the same workload with the DM basis and the reconstructor in bfloat16 (float32
    # sums and integrator): half the bytes of the dominant stream
    try:
        sysb = make_system(cfg_r, pas.PAS_BF16, pas.PAS_BF16, tuning, hist)
        try:
            rb = measure_loop(sysb, cfg, args, timed, barrier, flush, world, dist, peaks)
        finally:
            sysb.close()
        rb_wfe = rb.pop("wfe")
        extra["loop_bf16"] = {"steps_per_s": rb["value"], "ms_per_step": rb["ms_per_step"],
                              "dm_basis": "bf16", "reconstructor": "bf16 (per-row scale)",
                              "pwfs_frames_per_s": rb["pwfs_frames_per_s"], "kernel_ms": rb["kernel_ms"],
                              "roofline_by_kernel": rb["roofline_by_kernel"], "e2e": rb["e2e"],
                              "speedup_vs_fp32": rb["value"] / head["value"]}
        n = min(len(rb_wfe), len(head["wfe"]))
        if n:
            d = rb_wfe[:n] - head["wfe"][:n]
            extra["loop_bf16"]["wfe_diff_nm_rms"] = float(np.sqrt(np.mean(d * d)))
            extra["loop_bf16"]["wfe_nm_mean"] = float(np.mean(rb_wfe[n // 5:n]))
            extra["loop_bf16"]["wfe_nm_mean_fp32"] = float(np.mean(head["wfe"][n // 5:n]))
    except Exception as e:
        extra["loop_bf16"] = {"error": str(e)}
    if not args.no_extra:
        try:
            extra["scao_lbt_240px"], mlp_info = bench_lbt(args, timed, barrier, flush, world, dist, peaks,
                                                          no_mlp=args.no_mlp)
        except Exception as e:
            extra["scao_lbt_240px"] = {"error": str(e)}
        for key, kw in (("equal_wfe_bf16_vs_fp32", {}),
                        ("equal_wfe_bf16_vs_fp32_elt", {"workload": "scao_elt_480px", "n_modes": 1000})):
            try:
                extra[key] = bench_equal_wfe(timed, **kw)
            except Exception as e:
                extra[key] = {"error": str(e)}
        try:
            extra["other_workloads"] = bench_other_workloads(timed, peaks)
        except Exception as e:
            extra["other_workloads"] = {"error": str(e)}
        try:
            extra["shack_hartmann"] = bench_sh(timed)
        except Exception as e:
            extra["shack_hartmann"] = {"error": str(e)}
        try:
            extra["extended_source"] = bench_extended(timed)
        except Exception as e:
            extra["extended_source"] = {"error": str(e)}
        try:
            extra["monte_carlo_batch"] = bench_batch(timed)
        except Exception as e:
            extra["monte_carlo_batch"] = {"error": str(e)}
        try:
            extra["batched_workload"] = bench_batched_workload(timed)
        except Exception as e:
            extra["batched_workload"] = {"error": str(e)}

    clocks = sampler.stop() if sampler else None

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_for(cfg, args)

    line = {
        "metric": METRIC.format(workload=cfg.name), "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{cfg.name}: D={cfg.D} m, pupil {cfg.Np}^2 px, FFT {cfg.N}^2, "
                               f"{len(cfg.layers)} layers, {cfg.n_sub}x{cfg.n_sub} subaps, K={cfg.K}, "
                               f"R={cfg.mod_radius} l/D, {cfg.n_modes} modes, "
                               + (f"mag {cfg.magnitude} + {cfg.read_noise_e} e- RON" if cfg.magnitude is not None
                                  else "noiseless"),
                   "inputs": setup_note,
                   "l2": "flushed (256 MiB write + read) between timed steps", "recon": args.recon,
                   "parallelism": f"replicas x{world}", "graph": "whole step, CUDA graph"},
        "pwfs_frames_per_s": head["pwfs_frames_per_s"],
        "roofline": None if dom is None else {"bound": dom["bound"], "achieved": dom["achieved"],
                                               "peak": dom["peak"], "unit": dom["unit"], "frac": dom["frac"],
                                               "traffic": traffic, "kernel": dom["kernel"],
                                               "peak_source": dom["peak_source"]},
        "roofline_pwfs": pwfs_roof,
        "roofline_by_kernel": roof,
        "kernel_ms": head["kernel_ms"],
        "fp32_peak": fp32,
        "cpu_baseline": cpu,
        "e2e": head["e2e"],
        "gpu_launches": pas.PAS_LOOP_KERNELS * args.steps,
        "clocks": clocks,
        "learned_reconstructor": mlp_info,
        **extra,
        "setup_s": t_setup, "wall_timed_s": head["wall_timed_s"],
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
