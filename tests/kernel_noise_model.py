"""Float32 model of the detector-noise KERNEL's decisions (not the oracle).

This module restates, in NumPy float32 scalars, the exact arithmetic the CUDA
detector kernel uses to turn its Philox counter words into counts: a 24-bit
uniform, sequential-search inversion with the kernel's term recurrence below
lambda = 10, Hoermann's PTRS rejection (1993) in float32 above, Box-Muller read
noise added only to frames in photo-electrons. It exists so that GPU tests of the
loop machinery (integrators, hold steps, noisy closed loops) can feed the FP64
oracle loop the very counts the kernel drew and compare the two loops step by
step.

It is NOT a parity reference for the noise itself: it was written to agree with
the kernel. The noise is judged against the independent FP64 definition in
``oracle/noise.py`` statistically (``tests/test_gpu_noise_statistics.py``).
The Philox-4x32-10 generator is the published one (Salmon, Moraes, Dror, Shaw,
SC'11); its known-answer vectors are pinned in the oracle's tests.
"""
from __future__ import annotations

import math

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF
F32 = np.float32


def philox4x32_10(ctr, key):
    """Ten Philox-4x32 rounds: ctr = 4 x uint32, key = 2 x uint32 (Python ints)."""
    c0, c1, c2, c3 = [int(x) & MASK32 for x in ctr]
    k0, k1 = [int(x) & MASK32 for x in key]
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
    return c0, c1, c2, c3


def u01(x: int) -> np.float32:
    """Uniform in (0, 1), exact in float32."""
    return F32((x >> 8) + 0.5) * F32(2.0 ** -24)


def _block(seed: int, pixel: int, frame: int, blk: int):
    key = (seed & MASK32, (seed >> 32) & MASK32)
    return philox4x32_10((pixel, frame & MASK32, (frame >> 32) & MASK32, blk), key)


def poisson(lam, seed: int, pixel: int, frame: int) -> int:
    """Poisson(lam) drawn from the pixel's counter stream, decisions in float32."""
    lam = F32(lam)
    if not lam > 0:
        return 0
    w = _block(seed, pixel, frame, 0)
    if lam < F32(10.0):
        u = u01(w[2])
        p = np.exp(-lam)
        F = p
        k = 0
        while u > F and k < 256:
            k += 1
            p = F32(p * F32(lam * (F32(1.0) / F32(k))))
            Fn = F32(F + p)
            if Fn == F:        # the float32 CDF has stopped growing
                break
            F = Fn
        return k
    slam = np.sqrt(lam)
    loglam = np.log(lam)
    b = F32(F32(0.931) + F32(2.53) * slam)
    a = F32(F32(-0.059) + F32(0.02483) * b)
    invalpha = F32(F32(1.1239) + F32(1.1328) / (b - F32(3.4)))
    vr = F32(F32(0.9277) - F32(3.6224) / (b - F32(2.0)))
    blk = 0
    while blk < 64:
        if blk > 0:
            w = _block(seed, pixel, frame, blk)
        U = F32(u01(w[2]) - F32(0.5))
        V = u01(w[3])
        blk += 1
        us = F32(F32(0.5) - abs(U))
        k = np.floor((F32(2.0) * a / us + b) * U + lam + F32(0.43))
        if us >= F32(0.07) and V <= vr:
            return int(k)
        if k < 0 or (us < F32(0.013) and V > us):
            continue
        lhs = np.log(V) + np.log(invalpha) - np.log(a / (us * us) + b)
        rhs = -lam + k * loglam - F32(math.lgamma(float(F32(k) + F32(1.0))))
        if F32(lhs) <= F32(rhs):
            return int(k)
    return int(np.floor(lam + F32(0.5)))


def gaussian(seed: int, pixel: int, frame: int) -> np.float32:
    w = _block(seed, pixel, frame, 0)
    return F32(np.sqrt(F32(-2.0) * np.log(u01(w[0]))) * np.cos(F32(2.0 * math.pi) * u01(w[1])))


def apply_noise(frame_in: np.ndarray, photons_per_frame: float, n_pupil_px: int,
                read_noise_e: float, seed: int, frame_index: int) -> np.ndarray:
    """Noisy detector frame in photo-electrons (pixels in row-major order)."""
    flat = np.asarray(frame_in, dtype=np.float32).ravel()
    scale = F32(photons_per_frame / n_pupil_px)
    out = np.empty(flat.size, dtype=np.float64)
    for p, v in enumerate(flat):
        if photons_per_frame > 0:
            val = float(poisson(F32(v * scale), seed, p, frame_index))
            if read_noise_e > 0:
                val = float(F32(F32(val) + F32(read_noise_e) * gaussian(seed, p, frame_index)))
        else:
            val = float(v)
        out[p] = val
    return out.reshape(np.shape(frame_in))
