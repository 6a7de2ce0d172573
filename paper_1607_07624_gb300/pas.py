"""Thin ctypes binding of libpas.so (include/pas.h): argument marshalling only.

Every function keeps the C name; device buffers are passed as torch CUDA tensors
(their data_ptr), host buffers as numpy arrays. A non-zero status raises
PasError with the library's message. There is no fallback: if the library is not
built, importing this module raises ImportError.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libpas.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = C.CDLL(LIB_PATH)

PAS_OK, PAS_EINVAL, PAS_ENOMEM, PAS_ECUDA, PAS_ETIMEOUT, PAS_ESTATE = range(6)
PAS_FP32, PAS_BF16 = 0, 1
PAS_LOOP_KERNELS = 5          # kernels of one loop step (the header's define)
PAS_BATCH_PERSISTENT = 1      # pas_batch_create_ex flag
PAS_TAPS_AUTO, PAS_TAPS_TMA, PAS_TAPS_COPY = 0, 1, 2   # pas_atmo_set_tap_staging
STATUS_NAMES = {0: "PAS_OK", 1: "PAS_EINVAL", 2: "PAS_ENOMEM", 3: "PAS_ECUDA", 4: "PAS_ETIMEOUT",
                5: "PAS_ESTATE"}


class PasError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class pas_atmo_params(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("S", C.c_int32), ("Np", C.c_int32),
                ("vx", C.POINTER(C.c_double)), ("vy", C.POINTER(C.c_double))]


class pas_pyr_params(C.Structure):
    _fields_ = [("Np", C.c_int32), ("N", C.c_int32), ("K", C.c_int32), ("n_sub", C.c_int32),
                ("mod_radius", C.c_double), ("wavelength_nm", C.c_double), ("obs", C.c_double),
                ("local_norm", C.c_int32)]


class pas_pyr_tuning(C.Structure):
    _fields_ = [("rows_per_cta", C.c_int32), ("row_chunks", C.c_int32), ("col_groups", C.c_int32),
                ("col_split", C.c_int32)]


class pas_loop_stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("wfe_nm", C.c_double)]


vp = C.c_void_p
i32 = C.c_int32
i64 = C.c_int64
f64 = C.c_double
P = C.POINTER

_SIGS = {
    "pas_version": (C.c_int, []),
    "pas_ctx_create": (C.c_int, [vp, P(vp)]),
    "pas_ctx_destroy": (None, [vp]),
    "pas_ctx_set_stream": (C.c_int, [vp, vp]),
    "pas_ctx_synchronize": (C.c_int, [vp]),
    "pas_last_error": (C.c_char_p, [vp]),
    "pas_global_error": (C.c_char_p, []),
    "pas_debug_fail_alloc_after": (None, [C.c_int]),
    "pas_pupil_mask": (C.c_int, [C.c_int, f64, vp, P(i32)]),
    "pas_pupil_pixels": (C.c_int, [C.c_int, f64, vp, i32, P(i32)]),
    "pas_valid_subaps": (C.c_int, [C.c_int, f64, C.c_int, vp, i32, P(i32)]),
    "pas_atmo_create": (C.c_int, [vp, P(pas_atmo_params), vp, P(vp)]),
    "pas_atmo_advance": (C.c_int, [vp, i64, vp]),
    "pas_atmo_create_view": (C.c_int, [vp, vp, vp, P(vp)]),
    "pas_atmo_create_cone_view": (C.c_int, [vp, vp, vp, vp, P(vp)]),
    "pas_atmo_destroy": (None, [vp]),
    "pas_pyr_supported": (C.c_int, [C.c_int]),
    "pas_pyr_create": (C.c_int, [vp, P(pas_pyr_params), vp, i32, P(vp)]),
    "pas_pyr_create_extended": (C.c_int, [vp, P(pas_pyr_params), vp, i32, vp, vp, vp, i32, P(vp)]),
    "pas_pyr_n_valid": (i32, [vp]),
    "pas_pyr_get_valid": (C.c_int, [vp, vp, i32]),
    "pas_pyr_set_reference": (C.c_int, [vp, vp]),
    "pas_pyr_set_noise": (C.c_int, [vp, f64, f64, C.c_uint64, i64]),
    "pas_pyr_measure": (C.c_int, [vp, vp, vp, vp]),
    "pas_ccd_noise": (C.c_int, [vp, vp, vp, i32, f64, i32, f64, C.c_uint64, i64]),
    "pas_pyr_measure_static": (C.c_int, [P(pas_pyr_params), vp, i32, vp, vp, vp, vp, vp]),
    "pas_pyr_destroy": (None, [vp]),
    "pas_pyr_get_tuning": (C.c_int, [vp, P(pas_pyr_tuning)]),
    "pas_pyr_set_tuning": (C.c_int, [vp, P(pas_pyr_tuning)]),
    "pas_pyr_autotune": (C.c_int, [vp, vp, i32, P(pas_pyr_tuning)]),
    "pas_recon_create": (C.c_int, [vp, vp, i32, i32, C.c_int, P(vp)]),
    "pas_recon_apply": (C.c_int, [vp, vp, vp]),
    "pas_recon_destroy": (None, [vp]),
    "pas_dm_create": (C.c_int, [vp, vp, i32, i32, i32, f64, C.c_int, P(vp)]),
    "pas_dm_update": (C.c_int, [vp, vp, vp, vp, vp]),
    "pas_dm_residual": (C.c_int, [vp, vp, vp, vp]),
    "pas_dm_project": (C.c_int, [vp, vp, vp]),
    "pas_dm_destroy": (None, [vp]),
    "pas_loop_create": (C.c_int, [vp, vp, vp, vp, vp, vp, i32, i32, P(vp)]),
    "pas_loop_create_sh": (C.c_int, [vp, vp, vp, vp, vp, vp, i32, i32, P(vp)]),
    "pas_loop_step": (C.c_int, [vp, i32, P(pas_loop_stats)]),
    "pas_loop_step_eager": (C.c_int, [vp, i32]),
    "pas_loop_buffers": (C.c_int, [vp, P(vp), P(vp), P(vp), P(vp), P(vp), P(vp)]),
    "pas_loop_get_state": (C.c_int, [vp, P(i64), vp]),
    "pas_loop_set_state": (C.c_int, [vp, i64, vp]),
    "pas_loop_set_integration": (C.c_int, [vp, i32]),
    "pas_loop_destroy": (None, [vp]),
    "pas_loop_profile": (C.c_int, [vp, i32, vp, i32, P(i32)]),
    "pas_loop_kernel_name": (C.c_char_p, [i32]),
    "pas_mlp_create": (C.c_int, [vp, i32, vp, i32, P(vp)]),
    "pas_mlp_destroy": (None, [vp]),
    "pas_mlp_n_params": (i64, [vp]),
    "pas_mlp_set_params": (C.c_int, [vp, vp]),
    "pas_mlp_get_params": (C.c_int, [vp, vp]),
    "pas_mlp_set_norm": (C.c_int, [vp, vp, vp]),
    "pas_mlp_apply": (C.c_int, [vp, vp, vp]),
    "pas_mlp_forward": (C.c_int, [vp, i32, vp, vp]),
    "pas_mlp_gradients": (C.c_int, [vp, i32, vp, vp, vp, vp]),
    "pas_mlp_train": (C.c_int, [vp, vp, vp, i32, i32, vp, vp, i32, vp]),
    "pas_mlp_check": (C.c_int, [vp, P(C.c_uint32)]),
    "pas_mlp_pair": (C.c_int, [vp, vp, vp, C.c_float, vp, vp, vp]),
    "pas_loop_set_mlp": (C.c_int, [vp, vp]),
    "pas_gemm_bf16": (C.c_int, [vp, i32, i32, i32, vp, i32, vp, i32, vp, i32, i32, vp]),
    "pas_gemm_bf16_waits": (C.c_int, [vp, i32, i32, i32, vp, i32, vp, i32, vp, i32, i32, C.c_uint32, vp]),
    "pas_batch_create": (C.c_int, [vp, vp, i32, P(vp)]),
    "pas_batch_step": (C.c_int, [vp, i32]),
    "pas_batch_size": (i32, [vp]),
    "pas_batch_destroy": (None, [vp]),
    "pas_psf_create": (C.c_int, [vp, i32, i32, C.c_double, C.c_double, P(vp)]),
    "pas_psf_size": (i32, [vp]),
    "pas_psf_compute": (C.c_int, [vp, vp, vp, i32, vp]),
    "pas_psf_destroy": (None, [vp]),
    "pas_sh_create": (C.c_int, [vp, i32, i32, i32, C.c_double, C.c_double, vp, i32, P(vp)]),
    "pas_sh_n_valid": (i32, [vp]),
    "pas_sh_frame_side": (i32, [vp]),
    "pas_sh_get_valid": (C.c_int, [vp, vp, i32]),
    "pas_sh_set_reference": (C.c_int, [vp, vp]),
    "pas_sh_set_noise": (C.c_int, [vp, C.c_double, C.c_double, C.c_uint64, i64]),
    "pas_sh_measure": (C.c_int, [vp, vp, vp, vp]),
    "pas_sh_destroy": (None, [vp]),
    "pas_fp32_fma_probe": (C.c_int, [vp, vp, i32, i32, C.POINTER(C.c_int64)]),
    "pas_recon_check": (C.c_int, [vp, C.POINTER(C.c_uint32)]),
    "pas_batch_n_groups": (i32, [vp]),
    "pas_batch_kernels_per_step": (i32, [vp]),
    "pas_batch_check": (C.c_int, [vp, C.POINTER(C.c_uint32)]),
    "pas_batch_create_ex": (C.c_int, [vp, vp, i32, C.c_uint32, P(vp)]),
    "pas_atmo_tma": (i32, [vp]),
    "pas_loop_attach_camera": (C.c_int, [vp, vp, vp, vp, i32, i64]),
    "pas_atmo_set_tap_staging": (C.c_int, [vp, i32]),
    "pas_atmo_set_wait_limit": (C.c_int, [vp, C.c_uint32]),
    "pas_atmo_check": (C.c_int, [vp, C.POINTER(C.c_uint32)]),
    "pas_batch_n_persistent": (i32, [vp]),
    "pas_batch_n_residual_groups": (i32, [vp]),
    "pas_batch_persistent_geometry": (C.c_int, [vp, i32, P(i32)]),
    "pas_batch_set_wait_limit": (C.c_int, [vp, i64]),
    "pas_batch_probe_waits": (C.c_int, [vp, C.POINTER(C.c_uint32)]),
    "pas_calib_interaction_matrix": (C.c_int, [vp, vp, vp, C.c_double, vp]),
    "pas_pinv_f64": (C.c_int, [vp, vp, i32, i32, C.c_double, vp, vp, C.POINTER(i32), C.POINTER(i32)]),
    "pas_gemm_f64": (C.c_int, [vp, vp, C.c_int64, C.c_int64, vp, C.c_int64, C.c_int64, vp, i32, i32, i32, vp,
                               C.c_int64]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def _ptr(x):
    """Device pointer of a torch tensor / host pointer of a numpy array / None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _check(st: int, ctx=None):
    if st != PAS_OK:
        msg = (_lib.pas_last_error(ctx) if ctx else _lib.pas_global_error()) or b""
        raise PasError(st, msg.decode(errors="replace"))


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ------------------------------------------------------------------ functions

def pas_version() -> int:
    return _lib.pas_version()


def pas_ctx_create(stream=None):
    h = vp()
    _check(_lib.pas_ctx_create(_stream_handle(stream), C.byref(h)))
    return h


def pas_ctx_destroy(ctx):
    _lib.pas_ctx_destroy(ctx)


def pas_ctx_set_stream(ctx, stream):
    _check(_lib.pas_ctx_set_stream(ctx, _stream_handle(stream)), ctx)


def pas_ctx_synchronize(ctx):
    _check(_lib.pas_ctx_synchronize(ctx), ctx)


def pas_last_error(ctx) -> str:
    return (_lib.pas_last_error(ctx) or b"").decode()


def pas_debug_fail_alloc_after(n: int):
    _lib.pas_debug_fail_alloc_after(int(n))


def pas_pupil_mask(Np: int, obs: float) -> np.ndarray:
    m = np.zeros((Np, Np), dtype=np.uint8)
    n = i32()
    _check(_lib.pas_pupil_mask(Np, obs, m.ctypes.data, C.byref(n)))
    return m


def pas_pupil_pixels(Np: int, obs: float) -> np.ndarray:
    n = i32()
    _check(_lib.pas_pupil_pixels(Np, obs, None, 0, C.byref(n)))
    out = np.zeros(n.value, dtype=np.int32)
    _check(_lib.pas_pupil_pixels(Np, obs, out.ctypes.data, n.value, C.byref(n)))
    return out


def pas_valid_subaps(Np: int, obs: float, n_sub: int) -> np.ndarray:
    n = i32()
    _check(_lib.pas_valid_subaps(Np, obs, n_sub, None, 0, C.byref(n)))
    out = np.zeros(n.value, dtype=np.int32)
    _check(_lib.pas_valid_subaps(Np, obs, n_sub, out.ctypes.data, n.value, C.byref(n)))
    return out


def pas_atmo_create(ctx, n_layers, S, Np, vx, vy, d_screens):
    vx = np.ascontiguousarray(vx, dtype=np.float64)
    vy = np.ascontiguousarray(vy, dtype=np.float64)
    p = pas_atmo_params(n_layers, S, Np, vx.ctypes.data_as(P(C.c_double)), vy.ctypes.data_as(P(C.c_double)))
    h = vp()
    _check(_lib.pas_atmo_create(ctx, C.byref(p), _ptr(d_screens), C.byref(h)), ctx)
    return h


def pas_atmo_advance(atmo, ctx, step: int, d_opd):
    _check(_lib.pas_atmo_advance(atmo, int(step), _ptr(d_opd)), ctx)


def pas_atmo_create_view(atmo, ctx, ox, oy):
    """The same layers seen along another direction: per-layer footprint offsets [px]."""
    ox = np.ascontiguousarray(ox, dtype=np.float64)
    oy = np.ascontiguousarray(oy, dtype=np.float64)
    h = vp()
    _check(_lib.pas_atmo_create_view(atmo, ox.ctypes.data, oy.ctypes.data, C.byref(h)), ctx)
    return h


def pas_atmo_create_cone_view(atmo, ctx, ox, oy, scale=None):
    """The layers seen from a source at finite height: per-layer footprint offsets
    [px] and scales 1 - h/H (None: all 1)."""
    ox = np.ascontiguousarray(ox, dtype=np.float64)
    oy = np.ascontiguousarray(oy, dtype=np.float64)
    sp = None
    if scale is not None:
        scale = np.ascontiguousarray(scale, dtype=np.float64)
        sp = scale.ctypes.data
    h = vp()
    _check(_lib.pas_atmo_create_cone_view(atmo, ox.ctypes.data, oy.ctypes.data, sp, C.byref(h)), ctx)
    return h


def pas_atmo_destroy(atmo):
    _lib.pas_atmo_destroy(atmo)


def pas_pyr_supported(N: int) -> bool:
    return bool(_lib.pas_pyr_supported(N))


def pas_pyr_create(ctx, Np, N, K, n_sub, mod_radius, wavelength_nm, obs, valid=None, local_norm=0):
    p = pas_pyr_params(Np, N, K, n_sub, mod_radius, wavelength_nm, obs, local_norm)
    h = vp()
    if valid is not None:
        valid = np.ascontiguousarray(valid, dtype=np.int32)
        _check(_lib.pas_pyr_create(ctx, C.byref(p), valid.ctypes.data, valid.size, C.byref(h)), ctx)
    else:
        _check(_lib.pas_pyr_create(ctx, C.byref(p), None, 0, C.byref(h)), ctx)
    return h


def pas_pyr_create_extended(ctx, Np, N, K, n_sub, mod_radius, wavelength_nm, obs, ex, ey, w=None, valid=None,
                            local_norm=0):
    """The pyramid looking at an extended source: points at (ex, ey) lambda/D with
    relative intensities w (None: equal)."""
    p = pas_pyr_params(Np, N, K, n_sub, mod_radius, wavelength_nm, obs, local_norm)
    ex = np.ascontiguousarray(ex, dtype=np.float64)
    ey = np.ascontiguousarray(ey, dtype=np.float64)
    if ex.shape != ey.shape:
        raise ValueError("ex and ey differ in length")
    wp = None
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float64)
        if w.shape != ex.shape:
            raise ValueError("w and ex differ in length")
        wp = w.ctypes.data
    h = vp()
    vptr, nv = (None, 0)
    if valid is not None:
        valid = np.ascontiguousarray(valid, dtype=np.int32)
        vptr, nv = valid.ctypes.data, valid.size
    _check(_lib.pas_pyr_create_extended(ctx, C.byref(p), vptr, nv, ex.ctypes.data, ey.ctypes.data, wp, ex.size,
                                        C.byref(h)), ctx)
    return h


def pas_pyr_n_valid(pyr) -> int:
    return _lib.pas_pyr_n_valid(pyr)


def pas_pyr_get_valid(pyr, ctx) -> np.ndarray:
    n = _lib.pas_pyr_n_valid(pyr)
    out = np.zeros(n, dtype=np.int32)
    _check(_lib.pas_pyr_get_valid(pyr, out.ctypes.data, n), ctx)
    return out


def pas_pyr_set_reference(pyr, ctx, d_sn):
    _check(_lib.pas_pyr_set_reference(pyr, _ptr(d_sn)), ctx)


def pas_pyr_set_noise(pyr, ctx, photons, read_noise_e, seed, frame_index=0):
    _check(_lib.pas_pyr_set_noise(pyr, float(photons), float(read_noise_e), int(seed), int(frame_index)), ctx)


def pas_pyr_measure(pyr, ctx, d_opd, d_frame=None, d_slopes=None):
    _check(_lib.pas_pyr_measure(pyr, _ptr(d_opd), _ptr(d_frame), _ptr(d_slopes)), ctx)


def pas_pyr_measure_static(Np, N, K, n_sub, mod_radius, wavelength_nm, obs, d_opd, d_frame, d_slopes=None,
                           valid=None, d_sn=None, stream=None, local_norm=0):
    """Allocation-free pyramid measurement (no object, no device allocation).
    d_opd [Np, Np], d_frame [2 n_sub, 2 n_sub], d_slopes and d_sn [2 n_valid]: float32
    contiguous CUDA tensors (checked here: the C call cannot see their sizes)."""
    p = pas_pyr_params(Np, N, K, n_sub, mod_radius, wavelength_nm, obs, local_norm)
    if valid is not None:
        valid = np.ascontiguousarray(valid, dtype=np.int32)
        vptr, nv = valid.ctypes.data, valid.size
    else:
        vptr = None
        nv = pas_valid_subaps(Np, obs, n_sub).size if Np % max(n_sub, 1) == 0 else 0
    for name, t, n in (("d_opd", d_opd, Np * Np), ("d_frame", d_frame, 4 * n_sub * n_sub),
                       ("d_slopes", d_slopes, 2 * nv), ("d_sn", d_sn, 2 * nv)):
        if t is None:
            continue
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise PasError(PAS_EINVAL, f"pas_pyr_measure_static: {name} must be a contiguous float32 CUDA tensor")
        if t.numel() != n:
            raise PasError(PAS_EINVAL, f"pas_pyr_measure_static: {name} has {t.numel()} elements, needs {n}")
    nv = 0 if valid is None else nv
    _check(_lib.pas_pyr_measure_static(C.byref(p), vptr, nv, _ptr(d_sn), _ptr(d_opd), _ptr(d_frame),
                                       _ptr(d_slopes), _stream_handle(stream)))


def pas_ccd_noise(ctx, d_in, d_out, photons, n_pupil_pixels, read_noise_e, seed, frame_index):
    _check(_lib.pas_ccd_noise(ctx, _ptr(d_in), _ptr(d_out), d_in.numel(), float(photons),
                              int(n_pupil_pixels), float(read_noise_e), int(seed), int(frame_index)), ctx)


def pas_pyr_destroy(pyr):
    _lib.pas_pyr_destroy(pyr)


def _tuning_tuple(t):
    return (t.rows_per_cta, t.row_chunks, t.col_groups, t.col_split)


def pas_pyr_get_tuning(pyr, ctx):
    """(rows_per_cta, row_chunks, col_groups, col_split)."""
    t = pas_pyr_tuning()
    _check(_lib.pas_pyr_get_tuning(pyr, C.byref(t)), ctx)
    return _tuning_tuple(t)


def pas_pyr_set_tuning(pyr, ctx, rows_per_cta, row_chunks, col_groups, col_split=1):
    t = pas_pyr_tuning(rows_per_cta, row_chunks, col_groups, col_split)
    _check(_lib.pas_pyr_set_tuning(pyr, C.byref(t)), ctx)


def pas_pyr_autotune(pyr, ctx, d_opd, iters=5):
    t = pas_pyr_tuning()
    _check(_lib.pas_pyr_autotune(pyr, _ptr(d_opd), int(iters), C.byref(t)), ctx)
    return _tuning_tuple(t)


def pas_recon_create(ctx, R: np.ndarray, precision=PAS_FP32):
    R = np.ascontiguousarray(R, dtype=np.float32)
    h = vp()
    _check(_lib.pas_recon_create(ctx, R.ctypes.data, R.shape[0], R.shape[1], precision, C.byref(h)), ctx)
    return h


def pas_recon_apply(rec, ctx, d_slopes, d_dmodes):
    _check(_lib.pas_recon_apply(rec, _ptr(d_slopes), _ptr(d_dmodes)), ctx)


def pas_recon_destroy(rec):
    _lib.pas_recon_destroy(rec)


def pas_dm_create(ctx, M: np.ndarray, Np: int, obs: float, precision=PAS_FP32):
    M = np.ascontiguousarray(M, dtype=np.float32)
    h = vp()
    _check(_lib.pas_dm_create(ctx, M.ctypes.data, M.shape[0], M.shape[1], Np, obs, precision, C.byref(h)), ctx)
    return h


def pas_dm_update(dm, ctx, d_dmodes, d_gain, d_cmd, d_opd_dm):
    _check(_lib.pas_dm_update(dm, _ptr(d_dmodes), _ptr(d_gain), _ptr(d_cmd), _ptr(d_opd_dm)), ctx)


def pas_dm_residual(dm, ctx, d_opd_atm, d_cmd, d_opd_res):
    _check(_lib.pas_dm_residual(dm, _ptr(d_opd_atm), _ptr(d_cmd), _ptr(d_opd_res)), ctx)


def pas_dm_project(dm, ctx, d_opd, d_coeffs):
    _check(_lib.pas_dm_project(dm, _ptr(d_opd), _ptr(d_coeffs)), ctx)


def pas_dm_destroy(dm):
    _lib.pas_dm_destroy(dm)


def pas_loop_create(ctx, atmo, pyr, rec, dm, d_gain, delay=1, wfe_history=1):
    h = vp()
    _check(_lib.pas_loop_create(ctx, atmo, pyr, rec, dm, _ptr(d_gain), delay, wfe_history, C.byref(h)), ctx)
    return h


def pas_loop_create_sh(ctx, atmo, sh, rec, dm, d_gain, delay=1, wfe_history=1):
    h = vp()
    _check(_lib.pas_loop_create_sh(ctx, atmo, sh, rec, dm, _ptr(d_gain), delay, wfe_history, C.byref(h)), ctx)
    return h


def pas_loop_step(loop, ctx, n_steps=1, stats=False):
    if stats:
        s = pas_loop_stats()
        _check(_lib.pas_loop_step(loop, n_steps, C.byref(s)), ctx)
        return s.step, s.wfe_nm
    _check(_lib.pas_loop_step(loop, n_steps, None), ctx)
    return None


def pas_loop_step_eager(loop, ctx, n_steps=1):
    _check(_lib.pas_loop_step_eager(loop, n_steps), ctx)


def pas_loop_buffers(loop, ctx):
    ptrs = [vp() for _ in range(6)]
    _check(_lib.pas_loop_buffers(loop, *[C.byref(p) for p in ptrs]), ctx)
    names = ("opd_res", "frame", "slopes", "dmodes", "cmd", "wfe")
    return {n: p.value for n, p in zip(names, ptrs)}


def pas_loop_get_state(loop, ctx, n_modes: int, delay: int):
    step = i64()
    ring = np.zeros((delay, n_modes), dtype=np.float32)
    _check(_lib.pas_loop_get_state(loop, C.byref(step), ring.ctypes.data), ctx)
    return step.value, ring


def pas_loop_set_state(loop, ctx, step: int, ring: np.ndarray):
    ring = np.ascontiguousarray(ring, dtype=np.float32)
    _check(_lib.pas_loop_set_state(loop, int(step), ring.ctypes.data), ctx)


def pas_loop_set_integration(loop, ctx, n_int: int):
    """Detector steps per frame (1: a frame every step)."""
    _check(_lib.pas_loop_set_integration(loop, int(n_int)), ctx)


def pas_loop_destroy(loop):
    _lib.pas_loop_destroy(loop)


def pas_loop_profile(loop, ctx, n_steps=1):
    """Mean per-kernel duration [ms] of n_steps eager steps: {kernel name: ms}."""
    ms = np.zeros(16, dtype=np.float32)
    n = i32()
    _check(_lib.pas_loop_profile(loop, int(n_steps), ms.ctypes.data, ms.size, C.byref(n)), ctx)
    return {_lib.pas_loop_kernel_name(k).decode(): float(ms[k]) for k in range(n.value)}


def pas_loop_kernel_name(idx: int):
    r = _lib.pas_loop_kernel_name(int(idx))
    return r.decode() if r else None


def pas_mlp_create(ctx, sizes, max_batch: int):
    sz = np.ascontiguousarray(sizes, dtype=np.int32)
    h = vp()
    _check(_lib.pas_mlp_create(ctx, sz.size - 1, sz.ctypes.data, int(max_batch), C.byref(h)), ctx)
    return h


def pas_mlp_destroy(mlp):
    _lib.pas_mlp_destroy(mlp)


def pas_mlp_n_params(mlp) -> int:
    return int(_lib.pas_mlp_n_params(mlp))


def pas_mlp_set_params(mlp, ctx, params: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != pas_mlp_n_params(mlp):
        raise ValueError(f"expected {pas_mlp_n_params(mlp)} parameters, got {p.size}")
    _check(_lib.pas_mlp_set_params(mlp, p.ctypes.data), ctx)


def pas_mlp_get_params(mlp, ctx) -> np.ndarray:
    p = np.zeros(pas_mlp_n_params(mlp), dtype=np.float32)
    _check(_lib.pas_mlp_get_params(mlp, p.ctypes.data), ctx)
    return p


def pas_mlp_set_norm(mlp, ctx, mean: np.ndarray, inv_std: np.ndarray):
    m = np.ascontiguousarray(mean, dtype=np.float32)
    s = np.ascontiguousarray(inv_std, dtype=np.float32)
    _check(_lib.pas_mlp_set_norm(mlp, m.ctypes.data, s.ctypes.data), ctx)


def pas_mlp_apply(mlp, ctx, d_slopes, d_out):
    _check(_lib.pas_mlp_apply(mlp, _ptr(d_slopes), _ptr(d_out)), ctx)


def pas_mlp_forward(mlp, ctx, batch: int, d_S, d_out):
    _check(_lib.pas_mlp_forward(mlp, int(batch), _ptr(d_S), _ptr(d_out)), ctx)


def pas_mlp_gradients(mlp, ctx, batch: int, d_S, d_Y, d_grad) -> float:
    loss = C.c_float()
    _check(_lib.pas_mlp_gradients(mlp, int(batch), _ptr(d_S), _ptr(d_Y), _ptr(d_grad), C.byref(loss)), ctx)
    return float(loss.value)


def pas_mlp_train(mlp, ctx, d_S, d_Y, n_data: int, batch: int, d_idx, d_lr, n_steps: int, d_loss):
    _check(_lib.pas_mlp_train(mlp, _ptr(d_S), _ptr(d_Y), int(n_data), int(batch), _ptr(d_idx), _ptr(d_lr),
                              int(n_steps), _ptr(d_loss)), ctx)


def pas_mlp_check(mlp, ctx) -> int:
    f = C.c_uint32()
    _check(_lib.pas_mlp_check(mlp, C.byref(f)), ctx)
    return int(f.value)


def pas_mlp_pair(pyr, dm, ctx, d_opd, amp: float, d_work, d_slopes, d_coeffs):
    _check(_lib.pas_mlp_pair(pyr, dm, _ptr(d_opd), float(amp), _ptr(d_work), _ptr(d_slopes), _ptr(d_coeffs)), ctx)


def pas_loop_set_mlp(loop, ctx, mlp):
    _check(_lib.pas_loop_set_mlp(loop, mlp), ctx)


def pas_gemm_bf16(ctx, M, N, K, d_A, lda, d_B, ldb, d_C, ldc, d_err, tile_n=0):
    _check(_lib.pas_gemm_bf16(ctx, int(M), int(N), int(K), _ptr(d_A), int(lda), _ptr(d_B), int(ldb), _ptr(d_C),
                              int(ldc), int(tile_n), _ptr(d_err)), ctx)


def pas_gemm_bf16_waits(ctx, M, N, K, d_A, lda, d_B, ldb, d_C, ldc, d_err, wait_limit, tile_n=0):
    """pas_gemm_bf16 whose pipeline waits give up after wait_limit tries (0: at once);
    the bits of d_err (uint32 CUDA tensor) say which waits gave up."""
    _check(_lib.pas_gemm_bf16_waits(ctx, int(M), int(N), int(K), _ptr(d_A), int(lda), _ptr(d_B), int(ldb), _ptr(d_C),
                                    int(ldc), int(tile_n), int(wait_limit), _ptr(d_err)), ctx)


def pas_batch_create(ctx, loops):
    arr = (vp * len(loops))(*[l.value if isinstance(l, vp) else l for l in loops])
    h = vp()
    _check(_lib.pas_batch_create(ctx, arr, len(loops), C.byref(h)), ctx)
    return h


def pas_batch_create_ex(ctx, loops, flags=0):
    """pas_batch_create with flags (PAS_BATCH_PERSISTENT)."""
    arr = (vp * len(loops))(*[l.value if isinstance(l, vp) else l for l in loops])
    h = vp()
    _check(_lib.pas_batch_create_ex(ctx, arr, len(loops), int(flags), C.byref(h)), ctx)
    return h


def pas_batch_n_persistent(batch) -> int:
    return int(_lib.pas_batch_n_persistent(batch))


def pas_batch_persistent_geometry(batch, ctx, g):
    """Dict of persistent launch g's geometry."""
    h = (i32 * 8)()
    _check(_lib.pas_batch_persistent_geometry(batch, int(g), h), ctx)
    keys = ("N", "ctas", "threads", "smem_bytes", "rows_per_task", "sin_per_task", "rows_tasks", "columns_tasks")
    return dict(zip(keys, [int(v) for v in h]))


def pas_batch_n_residual_groups(batch) -> int:
    return int(_lib.pas_batch_n_residual_groups(batch))


def pas_batch_set_wait_limit(batch, ctx, polls):
    _check(_lib.pas_batch_set_wait_limit(batch, int(polls)), ctx)


def pas_batch_probe_waits(batch):
    """Run the wait diagnostic; returns (status, fault bits) without raising."""
    f = C.c_uint32()
    st = int(_lib.pas_batch_probe_waits(batch, C.byref(f)))
    return st, f.value


def pas_batch_step(batch, ctx, n_steps=1):
    _check(_lib.pas_batch_step(batch, int(n_steps)), ctx)


def pas_batch_size(batch) -> int:
    return int(_lib.pas_batch_size(batch))


def pas_batch_destroy(batch):
    _lib.pas_batch_destroy(batch)


def loaded_library_path() -> str:
    return LIB_PATH


# ------------------------------------------------------------------ PSF camera

def pas_psf_create(ctx, Np, nd, wavelength_nm, obs):
    h = vp()
    _check(_lib.pas_psf_create(ctx, int(Np), int(nd), float(wavelength_nm), float(obs), C.byref(h)), ctx)
    return h


def pas_psf_size(psf):
    return int(_lib.pas_psf_size(psf))


def pas_psf_compute(psf, ctx, d_opd, d_psf, accumulate=False, d_strehl=None):
    """PSF of the residual OPD d_opd into d_psf [N][N] (added when accumulate); the
    Strehl ratio into the float64 scalar d_strehl when given."""
    _check(_lib.pas_psf_compute(psf, _ptr(d_opd), _ptr(d_psf), 1 if accumulate else 0, _ptr(d_strehl)), ctx)


def pas_psf_destroy(psf):
    _lib.pas_psf_destroy(psf)


# ------------------------------------------------------ Shack-Hartmann WFS

def pas_sh_create(ctx, Np, n_sub, ovs, wavelength_nm, obs, valid=None):
    h = vp()
    v = None if valid is None else np.ascontiguousarray(valid, dtype=np.int32)
    _check(_lib.pas_sh_create(ctx, int(Np), int(n_sub), int(ovs), float(wavelength_nm), float(obs),
                              None if v is None else v.ctypes.data, 0 if v is None else int(v.size), C.byref(h)), ctx)
    return h


def pas_sh_n_valid(sh):
    return int(_lib.pas_sh_n_valid(sh))


def pas_sh_frame_side(sh):
    return int(_lib.pas_sh_frame_side(sh))


def pas_sh_get_valid(sh, ctx):
    out = np.zeros(pas_sh_n_valid(sh), dtype=np.int32)
    _check(_lib.pas_sh_get_valid(sh, out.ctypes.data, out.size), ctx)
    return out


def pas_sh_set_reference(sh, ctx, d_ref):
    _check(_lib.pas_sh_set_reference(sh, _ptr(d_ref)), ctx)


def pas_sh_set_noise(sh, ctx, photons, read_noise_e, seed, frame_index=0):
    _check(_lib.pas_sh_set_noise(sh, float(photons), float(read_noise_e), int(seed), int(frame_index)), ctx)


def pas_sh_measure(sh, ctx, d_opd, d_frame=None, d_slopes=None):
    _check(_lib.pas_sh_measure(sh, _ptr(d_opd), _ptr(d_frame), _ptr(d_slopes)), ctx)


def pas_sh_destroy(sh):
    _lib.pas_sh_destroy(sh)


def pas_fp32_fma_probe(d_sink, n_blocks, iters, stream=None) -> int:
    """Launch the FP32 FMA throughput probe (d_sink: float32 CUDA tensor of
    n_blocks * 256 elements); returns the launch's floating-point operations."""
    if d_sink.numel() < n_blocks * 256:
        raise PasError(PAS_EINVAL, "pas_fp32_fma_probe: d_sink too small")
    f = C.c_int64()
    _check(_lib.pas_fp32_fma_probe(_stream_handle(stream), _ptr(d_sink), int(n_blocks), int(iters), C.byref(f)))
    return int(f.value)


def _f64_cuda(name, t, numel=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise PasError(PAS_EINVAL, f"{name} must be a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise PasError(PAS_EINVAL, f"{name} has {t.numel()} elements, needs {numel}")


def pas_calib_interaction_matrix(ctx, dm, d_IM, amp_nm, n_modes, n_slopes, pyr=None, sh=None):
    """Push-pull interaction matrix on the GPU into d_IM (float64 CUDA tensor of
    shape (n_modes, n_slopes): row m is the IM's column m)."""
    _f64_cuda("d_IM", d_IM, n_modes * n_slopes)
    _check(_lib.pas_calib_interaction_matrix(pyr, sh, dm, float(amp_nm), _ptr(d_IM)), ctx)


def pas_pinv_f64(ctx, d_A, m, n, rcond, d_P):
    """FP64 pseudo-inverse of the m x n column-major d_A (a (n, m) row-major tensor)
    into d_P ((n, m) row-major = A^+). Returns (singular values, rank, sweeps)."""
    _f64_cuda("d_A", d_A, m * n)
    _f64_cuda("d_P", d_P, m * n)
    sv = np.zeros(n, dtype=np.float64)
    rank, sweeps = i32(), i32()
    _check(_lib.pas_pinv_f64(ctx, _ptr(d_A), int(m), int(n), float(rcond), _ptr(d_P), sv.ctypes.data,
                             C.byref(rank), C.byref(sweeps)), ctx)
    return sv, rank.value, sweeps.value


def pas_gemm_f64(ctx, X, sxi, sxj, Y, syk, syj, w, ni, nk, nj, Cout, ldc):
    """C[i*ldc + k] = sum_j X[i*sxi + j*sxj] w[j] Y[k*syk + j*syj] (FP64 CUDA tensors)."""
    for nm, t in (("X", X), ("Y", Y), ("C", Cout)) + ((("w", w),) if w is not None else ()):
        _f64_cuda(nm, t)
    _check(_lib.pas_gemm_f64(ctx, _ptr(X), int(sxi), int(sxj), _ptr(Y), int(syk), int(syj), _ptr(w), int(ni),
                             int(nk), int(nj), _ptr(Cout), int(ldc)), ctx)


def pas_recon_check(rec, ctx):
    """Raise PasError(PAS_ETIMEOUT) if a bounded wait of the reconstructor gave up."""
    f = C.c_uint32()
    _check(_lib.pas_recon_check(rec, C.byref(f)), ctx)
    return f.value


def pas_batch_n_groups(batch) -> int:
    """Groups of loops reconstructed together (shared bf16 reconstructor)."""
    return int(_lib.pas_batch_n_groups(batch))


def pas_batch_kernels_per_step(batch) -> int:
    return int(_lib.pas_batch_kernels_per_step(batch))


def pas_batch_check(batch, ctx):
    f = C.c_uint32()
    _check(_lib.pas_batch_check(batch, C.byref(f)), ctx)
    return f.value


def pas_atmo_tma(atmo) -> int:
    """1 when the residual's tap staging uses TMA boxes for this atmosphere."""
    return int(_lib.pas_atmo_tma(atmo))


def pas_atmo_set_wait_limit(atmo, ctx, tries):
    _check(_lib.pas_atmo_set_wait_limit(atmo, int(tries)), ctx)


def pas_atmo_check(atmo):
    """(status, fault bits) of the tap staging's waits, without raising."""
    f = C.c_uint32()
    st = int(_lib.pas_atmo_check(atmo, C.byref(f)))
    return st, f.value


def pas_atmo_set_tap_staging(atmo, ctx, mode):
    _check(_lib.pas_atmo_set_tap_staging(atmo, int(mode)), ctx)


def pas_loop_attach_camera(loop, ctx, psf, d_psf=None, d_sr=None, start_step=0):
    """The PSF camera inside the loop's step graph (psf None: detach). d_sr: float64
    CUDA tensor ring of Strehl ratios (entry t mod its length for step t) or None."""
    n = int(d_sr.numel()) if d_sr is not None else 1
    _check(_lib.pas_loop_attach_camera(loop, psf, _ptr(d_psf) if d_psf is not None else None,
                                       _ptr(d_sr) if d_sr is not None else None, n, int(start_step)), ctx)
