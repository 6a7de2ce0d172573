"""Oracle detector noise: Philox-4x32-10 counter RNG, photon and read-out noise.

Paper passage: the CCD object (Table 1 ``detector``: photon_noise, readout_noise,
readout_level, quantum_eff, bandw; ``wfs_source.magnitude``). The paper does not say
how noise is drawn. Readings:

  * photons per frame = F0 10^(-0.4 mag) (pi/4) D^2 (1 - obs^2) bandwidth QE dt;
    the expected count of detector pixel p is photons * I_p / n_pupil_pixels (the
    binned intensity sums to the pupil pixel count, Parseval);
  * counter-based RNG Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
    (seed low, seed high), counter = (pixel, frame low, frame high, block);
    u = (x + 0.5) 2^-32 in FP64;
  * read noise: Box-Muller on block 0 words 0, 1: sigma sqrt(-2 ln u0) cos(2 pi u1);
  * photon noise: Poisson by inversion (sequential search) on block 0 word 2 when
    lambda < 16, else the PTRS transformed rejection of Hoermann (1993) on pairs
    (word 2, word 3) of blocks 0, 1, 2, ...; all decisions in FP64.
"""
from __future__ import annotations

import math

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF


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


def u01(x: int) -> float:
    return (float(x) + 0.5) * 2.0 ** -32


def _block(seed: int, pixel: int, frame: int, blk: int):
    key = (seed & MASK32, (seed >> 32) & MASK32)
    return philox4x32_10((pixel, frame & MASK32, (frame >> 32) & MASK32, blk), key)


def poisson(lam: float, seed: int, pixel: int, frame: int) -> int:
    """Poisson(lam) drawn from the pixel's counter stream."""
    if lam <= 0.0:
        return 0
    w = _block(seed, pixel, frame, 0)
    if lam < 16.0:
        u = u01(w[2])
        k = 0
        p = math.exp(-lam)
        F = p
        while u > F and k < 1000:
            k += 1
            p *= lam / k
            F += p
        return k
    slam = math.sqrt(lam)
    loglam = math.log(lam)
    b = 0.931 + 2.53 * slam
    a = -0.059 + 0.02483 * b
    invalpha = 1.1239 + 1.1328 / (b - 3.4)
    vr = 0.9277 - 3.6224 / (b - 2.0)
    blk = 0
    while blk < 64:
        if blk > 0:
            w = _block(seed, pixel, frame, blk)
        U = u01(w[2]) - 0.5
        V = u01(w[3])
        blk += 1
        us = 0.5 - abs(U)
        k = math.floor((2.0 * a / us + b) * U + lam + 0.43)
        if us >= 0.07 and V <= vr:
            return int(k)
        if k < 0 or (us < 0.013 and V > us):
            continue
        if (math.log(V) + math.log(invalpha) - math.log(a / (us * us) + b)
                <= -lam + k * loglam - math.lgamma(k + 1.0)):
            return int(k)
    return int(math.floor(lam + 0.5))


def gaussian(seed: int, pixel: int, frame: int) -> float:
    w = _block(seed, pixel, frame, 0)
    return math.sqrt(-2.0 * math.log(u01(w[0]))) * math.cos(2.0 * math.pi * u01(w[1]))


def apply_noise(frame_in: np.ndarray, photons_per_frame: float, n_pupil_px: int,
                read_noise_e: float, seed: int, frame_index: int) -> np.ndarray:
    """Noisy detector frame in photo-electrons (pixels in row-major order)."""
    flat = np.asarray(frame_in, dtype=np.float64).ravel()
    scale = photons_per_frame / n_pupil_px
    out = np.empty_like(flat)
    for p, v in enumerate(flat):
        val = float(poisson(v * scale, seed, p, frame_index)) if photons_per_frame > 0 else v * scale
        if read_noise_e > 0:
            val += read_noise_e * gaussian(seed, p, frame_index)
        out[p] = val
    return out.reshape(np.shape(frame_in))
