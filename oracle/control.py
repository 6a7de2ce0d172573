"""Oracle control: integrator, residual wavefront error and the closed loop.

Paper passages: the integrator controller (Table 1 ``control``: delay, type 'INT',
int_gain), the run order of the loop (Table 2: atmo, prop, pyr, ccd, sc, rec, intc,
dm, ...) and the loop control object that triggers every processing object once
per simulation step (Sec. Structure; Sec. Build and run a simulation loop).
Readings:

  * the DM runs after the controller in a step and is a layer of the propagation,
    so the measurement at step t sees the command of step t - delay (delay 1 by
    default; the paper's example uses 2);
  * integrator c_t = c_{t-1} + g * (R s_t), with residual = atmosphere - M c;
  * residual wavefront error = RMS over pupil pixels of the residual OPD with its
    mean (piston) removed, in nm.
"""
from __future__ import annotations

from collections import deque

import numpy as np

from .atmosphere import atmo_opd, wind_velocity_px
from .modal import basis_to_grid
from .optics import pupil_mask, pwfs_intensity, detector_frame, pwfs_slopes


def integrator_step(c: np.ndarray, dc: np.ndarray, gain) -> np.ndarray:
    """c_t = c_{t-1} + g * dc (per-mode gain vector or scalar)."""
    return c + np.asarray(gain) * dc


def residual_wfe_nm(opd_res: np.ndarray, mask: np.ndarray) -> float:
    """sqrt(mean over pupil pixels of (opd - mean)^2)."""
    v = np.asarray(opd_res, dtype=np.float64)[mask]
    return float(np.sqrt(np.mean((v - v.mean()) ** 2)))


def residual_opd(opd_atm: np.ndarray, M: np.ndarray, c: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """mask * (atmosphere - M c) on the Np x Np grid."""
    return np.where(mask, opd_atm - basis_to_grid(M, c, mask), 0.0)


def closed_loop(cfg, screens_nm, M, R, sn, valid, n_steps, gain=None, delay=None,
                noise=None, use_fft=True, record=False, sensor=None, offsets_px=None, scales=None,
                n_int=1, slopes_of=None):
    """Run the SCAO loop for n_steps; returns dict with per-step WFE [nm] and the
    final command (and per-step slopes/commands if record). sensor: None for the
    modulated pyramid of cfg, else a callable (opd_res, t) -> (frame, slopes)
    already referenced (e.g. the Shack-Hartmann oracle); offsets_px: per-layer
    footprint offsets of an off-axis source (atmosphere.footprint_offsets_px);
    scales: per-layer footprint scales of a source at finite height;
    n_int: steps per detector frame of the pyramid (a detector integrating several
    simulation steps, Sec. Structure): each step's noiseless frame is added up and
    read out at the steps t with (t + 1) mod n_int = 0 as the window's mean, then the
    noise, the slopes and the integrator run; in between the command is held (the
    downstream objects follow the detector's rate) and the slopes keep their value;
    with a sensor callable, its noiseless frames are integrated and slopes_of(frame)
    gives the read-out frame's slopes."""
    gain = cfg.gain if gain is None else gain
    delay = cfg.delay if delay is None else delay
    mask = pupil_mask(cfg.Np, cfg.obs)
    vel = wind_velocity_px(cfg)
    n_m = M.shape[1]
    c = np.zeros(n_m)
    applied = deque([np.zeros(n_m) for _ in range(delay)], maxlen=delay)
    assert n_int >= 1 and (n_int == 1 or sensor is None or slopes_of is not None)
    wfe = np.empty(n_steps)
    hist = {"slopes": [], "cmd": [], "frame": []}
    acc = None
    s = np.zeros(2 * len(valid))
    frame = None
    for t in range(n_steps):
        opd_res = residual_opd(atmo_opd(screens_nm, vel, t, cfg.Np, offsets_px, scales), M, applied[0], mask)
        wfe[t] = residual_wfe_nm(opd_res, mask)
        readout = True
        if sensor is None:
            I = pwfs_intensity(opd_res, cfg.wavelength_nm, cfg.obs, cfg.N, cfg.K,
                               cfg.mod_radius, cfg.delta, use_fft=use_fft)
            f_t = detector_frame(I, cfg.n_sub)
            if frame is None:
                frame = np.zeros_like(f_t)       # the read-out frame, held between read-outs
            if n_int > 1:
                acc = f_t if acc is None else acc + f_t
                readout = (t + 1) % n_int == 0
            if readout:
                frame = f_t if n_int == 1 else acc / n_int
                acc = None
                if noise is not None:
                    frame = noise(frame, t)
                s = pwfs_slopes(frame, valid, cfg.n_sub, sn)
        elif n_int == 1:
            frame, s = sensor(opd_res, t)
        else:
            f_t = sensor(opd_res, t)[0]
            acc = f_t if acc is None else acc + f_t
            readout = (t + 1) % n_int == 0
            if frame is None:
                frame = np.zeros_like(f_t)
            if readout:
                frame = acc / n_int
                acc = None
                if noise is not None:
                    frame = noise(frame, t)
                s = slopes_of(frame)
        if readout:
            c = integrator_step(c, R @ s, gain)
        applied.append(c.copy())
        if record:
            hist["slopes"].append(s)
            hist["cmd"].append(c.copy())
            hist["frame"].append(frame)
    out = {"wfe": wfe, "cmd": c}
    if record:
        out.update({k: np.array(v) for k, v in hist.items()})
    return out
