"""SCAO system: the paper's processing-object chain built on libpas.so.

Mirrors the main file of the paper's example (Table 2): build the processing
objects from the parameters, connect them, calibrate (pupil indices, slope
reference, reconstruction matrix), then run the loop control. Device memory and
streams come from PyTorch; every per-step operation runs in libpas.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import calib
from . import pas as P


class DevView:
    """Zero-copy torch view of library-owned device memory."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}

    @staticmethod
    def tensor(ptr, shape, dtype="<f4"):
        return torch.as_tensor(DevView(ptr, shape, dtype), device="cuda")


class SCAOSystem:
    """Single-conjugate AO loop with a modulated pyramid, for one configuration.

    screens: float32 (L, S, S) OPD [nm] (host numpy or None: generated from the
    configuration's seeds); basis: float (n_pix, n_modes) (None: the configuration's
    basis, Zernike or KL);
    R: reconstruction matrix (None: calibrated by push-pull on the GPU);
    autotune: True (time the pyramid launch geometries on the GPU), False (library
    default) or (rows_per_cta, row_chunks, col_groups[, col_split]) to set one;
    sensor: "pyramid" (the configuration's modulated pyramid) or "sh" (a Shack-Hartmann
    sensor with the configuration's n_sub lenslets and spots of sh_ovs x the lenslet
    size, at the configuration's wavelength, with the same detector noise);
    source: None (on axis) or (rho_arcsec, phi_deg), an off-axis natural guide star:
    the loop sees each layer through a footprint moved by height x angle
    (pas_atmo_create_view), while `atmo_base` stays the on-axis atmosphere;
    (rho_arcsec, phi_deg, height_m) is a source at that height (a laser guide star):
    each footprint is also shrunk by 1 - h/H about the pupil centre (the cone
    effect, pas_atmo_create_cone_view);
    detector_steps: simulation steps per detector frame of the sensor (the detector's
    integration time over the loop's time step, pas_loop_set_integration): frames are
    read out, and the command updated, every detector_steps steps;
    extended_source: None (a point source) or (ex, ey[, w]): the pyramid sees an
    extended incoherent source of points at (ex, ey) lambda/D with intensities w
    (pas_pyr_create_extended; calib.disc_source builds a uniform disc)."""

    def __init__(self, cfg, screens=None, basis=None, R=None, recon_precision=P.PAS_FP32, dm_precision=P.PAS_FP32,
                 dm=None, rec=None,
                 noise=None, delay=None, wfe_history=4096, stream=None, build_loop=True,
                 autotune=True, sensor="pyramid", sh_ovs=2, source=None, detector_steps=1,
                 extended_source=None):
        from synth.inputs import layer_seeds, screen_white_noise
        self.cfg = cfg
        self.dev = torch.device("cuda")
        self.stream = stream or torch.cuda.current_stream()
        self.ctx = P.pas_ctx_create(self.stream)
        self.pix = P.pas_pupil_pixels(cfg.Np, cfg.obs)
        self.valid = P.pas_valid_subaps(cfg.Np, cfg.obs, cfg.n_sub)
        self.n_pix, self.n_valid = self.pix.size, self.valid.size
        # atmosphere
        if screens is None:
            noises = [screen_white_noise(cfg.S, s) for s in layer_seeds(cfg.seed, len(cfg.layers))]
            screens = calib.layer_screens(cfg, noises)
        self.d_screens = torch.as_tensor(np.ascontiguousarray(screens, dtype=np.float32)).to(self.dev)
        vel = calib.wind_shift_px(cfg)
        self.atmo_base = P.pas_atmo_create(self.ctx, len(cfg.layers), cfg.S, cfg.Np, vel[:, 0], vel[:, 1],
                                           self.d_screens)
        self.atmo = self.atmo_base
        self.source = source
        if source is not None:
            heights = [ly.height_m for ly in cfg.layers]
            off = np.array(calib.footprint_offsets_px(heights, source[0], source[1], cfg.dx),
                           dtype=np.float64).reshape(-1, 2)
            scale = calib.footprint_scales(heights, source[2]) if len(source) > 2 else None
            self.atmo = P.pas_atmo_create_cone_view(self.atmo_base, self.ctx, off[:, 0], off[:, 1], scale)
        # sensor + slope computer
        if sensor not in ("pyramid", "sh"):
            raise ValueError(f"sensor must be 'pyramid' or 'sh', not {sensor!r}")
        self.sensor = sensor
        self.pyr = self.sh = None
        if sensor == "sh":
            self.sh = P.pas_sh_create(self.ctx, cfg.Np, cfg.n_sub, sh_ovs, cfg.wavelength_nm, cfg.obs, self.valid)
            frame_side = P.pas_sh_frame_side(self.sh)
        else:
            if extended_source is None:
                self.pyr = P.pas_pyr_create(self.ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius,
                                            cfg.wavelength_nm, cfg.obs, self.valid)
            else:
                ex, ey = extended_source[0], extended_source[1]
                w = extended_source[2] if len(extended_source) > 2 else None
                self.pyr = P.pas_pyr_create_extended(self.ctx, cfg.Np, cfg.N, cfg.K, cfg.n_sub, cfg.mod_radius,
                                                     cfg.wavelength_nm, cfg.obs, ex, ey, w, self.valid)
            frame_side = cfg.n_det
        # DM
        self.basis_kind = "given"
        if basis is None:
            if cfg.basis == "kl" and cfg.n_modes <= calib.KL_MAX_MODES:
                basis = calib.kl_basis(cfg.Np, self.pix, cfg.n_modes, cfg.dx, cfg.r0_m, cfg.L0_m)
                self.basis_kind = "kl"
            elif cfg.n_modes > calib.HOST_GS_MAX_MODES:
                # the KL modes of this many Zernikes span the same space; with one gain
                # on every mode and an untruncated pseudo-inverse the loop does not
                # depend on the orthonormal basis chosen within that span
                basis = calib.zernike_basis_gpu(self.ctx, cfg.Np, self.pix, cfg.n_modes)
                self.basis_kind = "zernike (Cholesky QR on the GPU)"
            else:
                basis = calib.zernike_basis(cfg.Np, self.pix, cfg.n_modes)
                self.basis_kind = "zernike"
        self.basis = np.ascontiguousarray(basis, dtype=np.float32)
        self.n_modes = self.basis.shape[1]
        # a DM object holds only the basis: loops of one geometry may share one (dm=)
        self.own_dm = dm is None
        self.dm = P.pas_dm_create(self.ctx, self.basis, cfg.Np, cfg.obs, dm_precision) if dm is None else dm
        self.basis_bytes_per_el = 2.0 if dm_precision == P.PAS_BF16 else 4.0
        self.recon_bytes_per_el = 2.0 if recon_precision == P.PAS_BF16 else 4.0
        # buffers
        f32 = dict(device=self.dev, dtype=torch.float32)
        self.d_opd = torch.zeros(cfg.Np, cfg.Np, **f32)
        self.d_frame = torch.zeros(frame_side, frame_side, **f32)
        self.d_slopes = torch.zeros(2 * self.n_valid, **f32)
        self.d_sn = torch.zeros(2 * self.n_valid, **f32)
        # calibration: slope reference (flat wavefront, noiseless)
        set_ref = P.pas_sh_set_reference if self.sh else P.pas_pyr_set_reference
        set_ref(self.sh or self.pyr, self.ctx, None)
        self.measure(self.d_opd, reference=True)
        self.d_sn.copy_(self.d_slopes)
        set_ref(self.sh or self.pyr, self.ctx, self.d_sn)
        if R is None:
            R = self.calibrate_reconstructor()
        self.R = np.ascontiguousarray(R, dtype=np.float32)
        # a reconstructor object holds only R: loops of one system may share one (rec=),
        # and a batch then reconstructs them together with one tensor-core product
        self.own_rec = rec is None
        self.rec = P.pas_recon_create(self.ctx, self.R, recon_precision) if rec is None else rec
        self.d_gain = torch.full((self.n_modes,), cfg.gain, **f32)
        # launch geometry of the pyramid kernels, measured on the open-loop OPD
        self.tuning = P.pas_pyr_get_tuning(self.pyr, self.ctx) if self.pyr else None
        if self.sh:
            pass
        elif isinstance(autotune, (tuple, list)):
            P.pas_pyr_set_tuning(self.pyr, self.ctx, *autotune)
            self.tuning = P.pas_pyr_get_tuning(self.pyr, self.ctx)
        elif autotune:
            P.pas_atmo_advance(self.atmo, self.ctx, 0, self.d_opd)
            self.tuning = P.pas_pyr_autotune(self.pyr, self.ctx, self.d_opd, 5)
            self.d_opd.zero_()
        if noise is None and cfg.magnitude is not None:
            noise = (calib.detector_photons(cfg), cfg.read_noise_e, cfg.seed)
        if noise is not None:
            set_noise = P.pas_sh_set_noise if self.sh else P.pas_pyr_set_noise
            set_noise(self.sh or self.pyr, self.ctx, noise[0], noise[1], noise[2], 0)
        self.delay = cfg.delay if delay is None else delay
        self.loop = None
        if build_loop:
            if self.sh:
                self.loop = P.pas_loop_create_sh(self.ctx, self.atmo, self.sh, self.rec, self.dm, self.d_gain,
                                                 self.delay, wfe_history)
            else:
                self.loop = P.pas_loop_create(self.ctx, self.atmo, self.pyr, self.rec, self.dm, self.d_gain,
                                              self.delay, wfe_history)
            if detector_steps != 1:
                P.pas_loop_set_integration(self.loop, self.ctx, detector_steps)
            b = P.pas_loop_buffers(self.loop, self.ctx)
            self.wfe_history = wfe_history
            self.loop_opd = DevView.tensor(b["opd_res"], (cfg.Np, cfg.Np))
            self.loop_frame = DevView.tensor(b["frame"], (frame_side, frame_side))
            self.loop_slopes = DevView.tensor(b["slopes"], (2 * self.n_valid,))
            self.loop_dmodes = DevView.tensor(b["dmodes"], (self.n_modes,))
            self.loop_cmd = DevView.tensor(b["cmd"], (self.n_modes,))
            self.loop_wfe = DevView.tensor(b["wfe"], (wfe_history,), "<f8")

    # ---------------------------------------------------------------- steps
    def measure(self, d_opd, reference=False):
        """opd -> (frame, slopes) through the sensor (device tensors)."""
        if self.sh:
            P.pas_sh_measure(self.sh, self.ctx, d_opd, self.d_frame, self.d_slopes)
        else:
            P.pas_pyr_measure(self.pyr, self.ctx, d_opd, self.d_frame, self.d_slopes)
        return self.d_frame, self.d_slopes

    def calibrate_reconstructor(self, amp_nm=None, rcond=1e-3):
        """Push-pull interaction matrix measured by the GPU sensor
        (pas_calib_interaction_matrix) and its FP64 pseudo-inverse by one-sided Jacobi
        SVD on the GPU (pas_pinv_f64); singular values below rcond x the largest are
        dropped. Keeps IM (n_slopes x n_modes, host FP64) and its singular values."""
        amp = self.cfg.pushpull_nm if amp_nm is None else amp_nm
        ns, nm = 2 * self.n_valid if self.pyr else P.pas_sh_n_valid(self.sh) * 2, self.n_modes
        d_IM = torch.empty(nm, ns, device=self.dev, dtype=torch.float64)   # row m = IM column m
        P.pas_calib_interaction_matrix(self.ctx, self.dm, d_IM, amp, nm, ns, pyr=self.pyr, sh=self.sh)
        d_R = torch.empty(nm, ns, device=self.dev, dtype=torch.float64)
        self.im_singular_values, self.im_rank, self.pinv_sweeps = P.pas_pinv_f64(self.ctx, d_IM, ns, nm, rcond, d_R)
        self.IM = d_IM.t().cpu().numpy()
        return d_R.cpu().numpy()

    def step(self, n=1, stats=False):
        cam = getattr(self, "camera", None)
        if cam is None or getattr(self, "_cam_in_graph", False):
            out = P.pas_loop_step(self.loop, self.ctx, n, stats)
            self._t = getattr(self, "_t", 0) + n
            return out
        # with a camera: after each loop step from its start step on, the PSF of that
        # step's residual is added to int_psf and its Strehl ratio written to sr[t mod len]
        t = getattr(self, "_t", 0)
        sci = self._cmd_queue is not None
        for _ in range(n):
            applied = self._cmd_queue.popleft() if sci else None   # command applied at step t
            P.pas_loop_step(self.loop, self.ctx, 1, False)
            if t >= self.camera_start:
                opd = self.loop_opd
                if sci:   # on-axis residual: the base atmosphere at t minus the applied DM shape
                    P.pas_atmo_advance(self.atmo_base, self.ctx, t, self._sci_atm)
                    P.pas_dm_residual(self.dm, self.ctx, self._sci_atm, applied, self._sci_res)
                    opd = self._sci_res
                slot = self.sr.data_ptr() + 8 * (t % self.sr.numel())
                P.pas_psf_compute(cam, self.ctx, opd, self.int_psf, True, slot)
            if sci:
                self._cmd_queue.append(self.loop_cmd.clone())
            t += 1
        self._t = t
        return P.pas_loop_step(self.loop, self.ctx, 0, True) if stats else None

    # ---------------------------------------------------------------- camera
    def attach_camera(self, nd=8, wavelength_nm=1650.0, start_step=0, sr_history=None, direction="science",
                      in_graph=True):
        """PSF camera on the loop's residual (Table 1 camera: imaging wavelength,
        padding nd, integration start): from loop step `start_step` on, every step's
        PSF ([N][N], N = nd Np, peak 1 for a flat wavefront at (N/2, N/2)) is added to
        `int_psf` and its Strehl ratio written to `sr` (float64 ring; entry t mod its
        length belongs to step t). direction: "science" (on axis) or "wfs" (the guide
        star's direction); they differ only with an off-axis source. Where the camera
        images the loop's own residual (on axis, or direction "wfs") it runs inside the
        step graph (in_graph, pas_loop_attach_camera); otherwise one call per step after
        it. Returns N."""
        if direction not in ("science", "wfs"):
            raise ValueError(f"direction must be 'science' or 'wfs', not {direction!r}")
        self.detach_camera()
        self._cmd_queue = None
        if direction == "science" and self.source is not None:
            from collections import deque
            f32 = dict(device=self.dev, dtype=torch.float32)
            self._sci_atm = torch.zeros(self.cfg.Np, self.cfg.Np, **f32)
            self._sci_res = torch.zeros(self.cfg.Np, self.cfg.Np, **f32)
            t0, ring = self.get_state()
            # the command applied at steps t0, t0+1, ...: ring slot (t mod delay) before step t
            self._cmd_queue = deque(torch.as_tensor(ring[(t0 + k) % self.delay]).to(self.dev)
                                    for k in range(self.delay))
            self._t = t0
        self.camera = P.pas_psf_create(self.ctx, self.cfg.Np, nd, wavelength_nm, self.cfg.obs)
        N = P.pas_psf_size(self.camera)
        self.int_psf = torch.zeros(N, N, device=self.dev, dtype=torch.float32)
        self.sr = torch.zeros(sr_history or getattr(self, "wfe_history", 1024), device=self.dev,
                              dtype=torch.float64)
        self.camera_start = int(start_step)
        self._cam_in_graph = bool(in_graph) and self._cmd_queue is None and self.loop is not None
        if self._cam_in_graph:
            P.pas_loop_attach_camera(self.loop, self.ctx, self.camera, self.int_psf, self.sr, self.camera_start)
        return N

    def detach_camera(self):
        cam = getattr(self, "camera", None)
        if cam is not None:
            if getattr(self, "_cam_in_graph", False) and self.loop is not None:
                P.pas_loop_attach_camera(self.loop, self.ctx, None)
            torch.cuda.synchronize()
            P.pas_psf_destroy(cam)
        self.camera = None
        self._cam_in_graph = False
        self._cmd_queue = None

    def step_eager(self, n=1):
        P.pas_loop_step_eager(self.loop, self.ctx, n)
        self._t = getattr(self, "_t", 0) + n

    def wfe_nm(self, n_steps):
        """Per-step residual WFE [nm] of the first n_steps (n_steps <= history)."""
        torch.cuda.synchronize()
        return self.loop_wfe[:n_steps].cpu().numpy().copy()

    def get_state(self):
        return P.pas_loop_get_state(self.loop, self.ctx, self.n_modes, self.delay)

    def set_state(self, step, ring):
        P.pas_loop_set_state(self.loop, self.ctx, step, ring)
        self._t = int(step)

    def close(self):
        if getattr(self, "ctx", None):
            self.detach_camera()
        dm = getattr(self, "dm", None) if getattr(self, "own_dm", True) else None
        rec = getattr(self, "rec", None) if getattr(self, "own_rec", True) else None
        for h, f in ((getattr(self, "loop", None), P.pas_loop_destroy), (rec, P.pas_recon_destroy),
                     (dm, P.pas_dm_destroy), (getattr(self, "pyr", None), P.pas_pyr_destroy),
                     (getattr(self, "sh", None), P.pas_sh_destroy),
                     (getattr(self, "atmo", None) if getattr(self, "source", None) is not None else None,
                      P.pas_atmo_destroy),
                     (getattr(self, "atmo_base", None), P.pas_atmo_destroy)):
            if h:
                f(h)
        self.loop = self.rec = self.dm = self.pyr = self.sh = self.atmo = self.atmo_base = None
        if getattr(self, "ctx", None):
            torch.cuda.synchronize()
            P.pas_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
