"""Learned nonlinear reconstructor: training pairs from the simulator, training
on the tensor cores, use in the closed loop with the linear reconstructor as
fallback.

The paper's reconstructor is linear (Table 1 modalrec); a multilayer perceptron
from slopes to modal coefficients is an extension built on the same objects.
Readings made here:
  * Training phases model the residual of a working closed loop without
    running one: an open-loop OPD of the simulated atmosphere at a random time,
    minus the fraction (1 - eps) of its projection on the DM modes, so the
    uncorrectable part beyond the modes stays whole and the modal part keeps a
    fraction eps (log-uniform in eps_range, one value per phase) as temporal
    error. Seeing enters as the factor (r0 / r0_config)^(-5/6) on the OPD, with
    r0 uniform in r0_range; each phase gives one pair per amplitude factor a in
    `amps`: slopes of the scaled phase (noiseless pyramid, reference
    subtracted) and its modal projection (1/n_pix) M^T (scaled phase).
  * Inputs are standardised per slope with the training-set mean and standard
    deviation; targets are divided by one global scale (their RMS) during
    training and the output layer is rescaled afterwards, so the network
    predicts coefficients in nm and the loss is the plain MSE up to a constant.
  * Adam with a cosine learning-rate schedule, He-normal initial weights,
    zero biases.
Every arithmetic step of training and inference runs in the library's kernels;
the dataset statistics and the schedule are set-up computations on the host or
in PyTorch.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import pas as P
from synth.inputs import rng


def he_normal_params(sizes, seed: int) -> np.ndarray:
    """Packed float32 parameters: W_l ~ N(0, 2 / fan_in), b_l = 0."""
    g = rng(seed)
    parts = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        parts.append((g.standard_normal((b, a)) * math.sqrt(2.0 / a)).ravel())
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


def cosine_lr(lr_max: float, n_steps: int, warmup: int = 0) -> np.ndarray:
    t = np.arange(n_steps, dtype=np.float64)
    lr = lr_max * 0.5 * (1.0 + np.cos(np.pi * t / max(n_steps, 1)))
    if warmup > 0:
        lr[:warmup] *= (t[:warmup] + 1) / warmup
    return lr.astype(np.float32)


class MLPReconstructor:
    """The network object of the C ABI plus its training bookkeeping."""

    def __init__(self, ctx, sizes, max_batch: int = 1024, seed: int = 0):
        self.ctx = ctx
        self.sizes = [int(s) for s in sizes]
        self.max_batch = int(max_batch)
        self.h = P.pas_mlp_create(ctx, self.sizes, self.max_batch)
        self.set_params(he_normal_params(self.sizes, seed))
        self.mean = np.zeros(self.sizes[0], np.float32)
        self.inv_std = np.ones(self.sizes[0], np.float32)
        self.y_scale = 1.0

    # ------------------------------------------------------------ parameters
    def set_params(self, p: np.ndarray):
        P.pas_mlp_set_params(self.h, self.ctx, p)

    def get_params(self) -> np.ndarray:
        return P.pas_mlp_get_params(self.h, self.ctx)

    def set_norm(self, mean, inv_std):
        self.mean = np.asarray(mean, np.float32)
        self.inv_std = np.asarray(inv_std, np.float32)
        P.pas_mlp_set_norm(self.h, self.ctx, self.mean, self.inv_std)

    def _scale_output_layer(self, f: float):
        p = self.get_params()
        n_last = self.sizes[-1] * self.sizes[-2] + self.sizes[-1]
        p[-n_last:] *= np.float32(f)
        self.set_params(p)

    # ------------------------------------------------------------ training
    def fit(self, d_S, d_Y, epochs: int = 10, batch: int = 1024, lr: float = 1e-3, seed: int = 0,
            warmup: int = 0, renorm: bool = True):
        """Train on device tensors d_S [n][n_in], d_Y [n][n_out] (float32).
        renorm: take the input standardisation and target scale from this data
        set (False keeps those of the previous fit, for continued training).
        Returns the per-step loss (in units of the target scale squared)."""
        n = int(d_S.shape[0])
        batch = min(batch, n, self.max_batch)
        if renorm:
            # set-up: standardisation and target scale from the training set
            mean = d_S.mean(0)
            std = d_S.std(0).clamp_min(1e-6)
            self.set_norm(mean.cpu().numpy(), (1.0 / std).cpu().numpy())
            self.y_scale = float(d_Y.pow(2).mean().sqrt().item()) or 1.0
        d_Yn = (d_Y / self.y_scale).contiguous()
        per_epoch = n // batch
        total = epochs * per_epoch
        g = rng(seed)
        idx = np.concatenate([g.permutation(n)[:per_epoch * batch] for _ in range(epochs)]).astype(np.int32)
        d_idx = torch.as_tensor(idx, device=d_S.device)
        d_lr = torch.as_tensor(cosine_lr(lr, total, warmup), device=d_S.device)
        d_loss = torch.zeros(total, device=d_S.device)
        # parameters currently predict nm: move the output layer to the training units
        self._scale_output_layer(1.0 / self.y_scale)
        P.pas_mlp_train(self.h, self.ctx, d_S.contiguous(), d_Yn, n, batch, d_idx, d_lr, total, d_loss)
        P.pas_mlp_check(self.h, self.ctx)
        self._scale_output_layer(self.y_scale)
        return d_loss.cpu().numpy()

    # ------------------------------------------------------------ inference
    def forward(self, d_S):
        """Batched inference (tensor cores): d_S [B][n_in] -> [B][n_out] device tensor."""
        B = int(d_S.shape[0])
        out = torch.empty(B, self.sizes[-1], device=d_S.device)
        for b0 in range(0, B, self.max_batch):
            b1 = min(B, b0 + self.max_batch)
            P.pas_mlp_forward(self.h, self.ctx, b1 - b0, d_S[b0:b1].contiguous(), out[b0:b1])
        return out

    def check(self) -> int:
        return P.pas_mlp_check(self.h, self.ctx)

    def close(self):
        if self.h:
            torch.cuda.synchronize()
            P.pas_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate_pairs(system, n_pairs: int, amps=(0.5, 1.0, 2.0), r0_range=(0.05, 0.2), eps_range=(0.03, 0.6),
                   seed: int = 0):
    """(slopes, coefficients) pairs of modelled closed-loop residual phases of
    `system`'s atmosphere (see the module docstring). The system's pyramid must
    be noiseless. Returns device tensors S [n_pairs][2 n_valid], Y [n_pairs][n_modes];
    consecutive pairs share a phase and differ by the amplitude factor."""
    cfg = system.cfg
    dev = system.d_screens.device
    S = torch.empty(n_pairs, 2 * system.n_valid, device=dev)
    Y = torch.empty(n_pairs, system.n_modes, device=dev)
    work = torch.empty(cfg.Np * cfg.Np + cfg.n_det ** 2, device=dev)
    opd = torch.empty(cfg.Np, cfg.Np, device=dev)
    res = torch.empty(cfg.Np, cfg.Np, device=dev)
    c = torch.empty(system.n_modes, device=dev)
    g = rng(seed)
    lo, hi = np.log(eps_range[0]), np.log(eps_range[1])
    k = 0
    while k < n_pairs:
        P.pas_atmo_advance(system.atmo, system.ctx, int(g.integers(0, 1 << 30)), opd)
        P.pas_dm_project(system.dm, system.ctx, opd, c)
        c.mul_(float(1.0 - np.exp(g.uniform(lo, hi))))
        P.pas_dm_residual(system.dm, system.ctx, opd, c, res)
        f = float((g.uniform(*r0_range) / cfg.r0_m) ** (-5.0 / 6.0))
        for a in amps:
            if k >= n_pairs:
                break
            P.pas_mlp_pair(system.pyr, system.dm, system.ctx, res, a * f, work, S[k], Y[k])
            k += 1
    return S, Y


def collect_on_policy(system, mlp: MLPReconstructor | None, n_pairs: int, r0_range=(0.05, 0.2),
                      max_steps: int = 1500, every: int = 2, stop_wfe_nm: float | None = None, seed: int = 0):
    """Pairs from the states the loop actually visits with reconstructor `mlp`
    (None: linear), for data-set aggregation: per run the screens are scaled to
    a random r0 and the loop starts at a random time from a zero command; every
    `every` steps the residual OPD gives one pair (amplitude 1). A run ends after
    max_steps or once the step's WFE exceeds stop_wfe_nm * (r0 / r0_config)^(-5/6).
    Leaves the loop at step 0 with the linear reconstructor and the original
    screens. Returns S, Y as generate_pairs."""
    cfg = system.cfg
    dev = system.d_screens.device
    S = torch.empty(n_pairs, 2 * system.n_valid, device=dev)
    Y = torch.empty(n_pairs, system.n_modes, device=dev)
    work = torch.empty(cfg.Np * cfg.Np + cfg.n_det ** 2, device=dev)
    base = system.d_screens.clone()
    zeros = np.zeros((system.delay, system.n_modes), np.float32)
    g = rng(seed)
    k = 0
    P.pas_loop_set_mlp(system.loop, system.ctx, mlp.h if mlp else None)
    try:
        while k < n_pairs:
            f = float((g.uniform(*r0_range) / cfg.r0_m) ** (-5.0 / 6.0))
            system.d_screens.copy_(base * f)
            system.set_state(int(g.integers(0, 1 << 30)), zeros)
            t = 0
            while t < max_steps and k < n_pairs:
                st = system.step(every, stats=stop_wfe_nm is not None)
                t += every
                P.pas_mlp_pair(system.pyr, system.dm, system.ctx, system.loop_opd, 1.0, work, S[k], Y[k])
                k += 1
                if stop_wfe_nm is not None and st[1] > stop_wfe_nm * f:
                    break
        if mlp is not None:
            mlp.check()
    finally:
        P.pas_loop_set_mlp(system.loop, system.ctx, None)
        system.d_screens.copy_(base)
        system.set_state(0, zeros)
    return S, Y


def run_loop(system, n_steps: int, mlp: MLPReconstructor | None = None, check_every: int = 250):
    """Closed loop for n_steps from the loop's current state, with the network
    (or the linear reconstructor when mlp is None). The network is checked every
    `check_every` steps; after a non-finite output the loop falls back to the
    linear reconstructor for the rest of the run. Returns (per-step WFE [nm],
    step of the fallback or None); needs n_steps <= the loop's WFE history."""
    P.pas_loop_set_mlp(system.loop, system.ctx, mlp.h if mlp else None)
    step0, _ = system.get_state()
    fallback = None
    done = 0
    try:
        while done < n_steps:
            n = min(check_every, n_steps - done)
            system.step(n)
            done += n
            if mlp is not None and fallback is None and mlp.check():
                fallback = step0 + done
                P.pas_loop_set_mlp(system.loop, system.ctx, None)
    finally:
        P.pas_loop_set_mlp(system.loop, system.ctx, None)
    torch.cuda.synchronize()
    hist = system.loop_wfe.cpu().numpy()
    steps = np.arange(step0, step0 + n_steps)
    return hist[steps % system.wfe_history].copy(), fallback
