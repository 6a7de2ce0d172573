"""Oracle detector noise in FP64: Philox-4x32-10 counter RNG, photon and read-out noise.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper passage: the CCD object (Table 1 ``detector``: photon_noise, readout_noise,
readout_level, quantum_eff, bandw; ``wfs_source.magnitude``). The paper does not say
how noise is drawn. Readings:

  * a frame in photo-electrons exists only when the detector receives photons
    (photons per frame > 0); the expected count of detector pixel p is
    lambda_p = photons * I_p / n_pupil_pixels (the binned intensity sums to the pupil
    pixel count, Parseval). With photons <= 0 the frame stays noiseless intensity;
  * pixel p of frame t draws from its own counter stream of Philox-4x32-10
    (Salmon, Moraes, Dror, Shaw, SC'11): key = (seed low, seed high), counter =
    (p, t low, t high, block); a 32-bit word x gives the FP64 uniform
    u = (x + 1/2) 2^-32 in (0, 1);
  * photon noise: the Poisson(lambda_p) count is the inverse of the Poisson
    cumulative distribution at u = uniform(block 0, word 2): the smallest k with
    P(X <= k) >= u (sampling by inversion; the CDF is the regularised incomplete
    gamma function Q(k + 1, lambda), scipy's ``pdtr``, in FP64);
  * read noise, whenever its sigma is > 0 (also on pixels that receive no light):
    sigma * N(0, 1) with N(0, 1) = sqrt(-2 ln u0) cos(2 pi u1) (Box-Muller, 1958),
    u0, u1 = uniforms of block 0 words 0 and 1.

Nothing here follows the GPU kernel's arithmetic: its float32 decisions (24-bit
uniforms, a rejection sampler above lambda = 10) draw from the same law, and the
GPU's frames are judged against this definition statistically.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import gammaln, pdtr

# Philox-4x32-10 constants (Salmon et al., SC'11): round multipliers and Weyl key
# increments (the golden ratio and sqrt(3) - 1 in 32-bit fixed point).
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


def uniform(x: int) -> float:
    """FP64 uniform in (0, 1) from a 32-bit word."""
    return (float(x) + 0.5) * 2.0 ** -32


def counter_words(seed: int, pixel: int, frame: int, block: int = 0):
    key = (seed & MASK32, (seed >> 32) & MASK32)
    return philox4x32_10((pixel, frame & MASK32, (frame >> 32) & MASK32, block), key)


def poisson_pmf(k, lam):
    """P(X = k) for X ~ Poisson(lam), FP64 (lam > 0, k >= 0 integers)."""
    k = np.asarray(k, dtype=np.float64)
    return np.exp(k * math.log(lam) - lam - gammaln(k + 1.0))


def poisson_inverse_cdf(u, lam):
    """Smallest integer k >= 0 with P(X <= k) >= u, X ~ Poisson(lam) (elementwise;
    lam > 0, 0 < u < 1). The search starts at floor(lam) and walks to the boundary."""
    u = np.asarray(u, dtype=np.float64)
    lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), u.shape)
    k = np.floor(lam)
    # down: while P(X <= k - 1) >= u
    while True:
        m = (k > 0) & (pdtr(np.maximum(k - 1, 0), lam) >= u)
        if not m.any():
            break
        k = np.where(m, k - 1, k)
    # up: while P(X <= k) < u
    while True:
        m = pdtr(k, lam) < u
        if not m.any():
            break
        k = np.where(m, k + 1, k)
    return k.astype(np.int64)


def poisson(lam: float, seed: int, pixel: int, frame: int) -> int:
    """Poisson(lam) count of one pixel by inversion of its block-0 word-2 uniform."""
    if not lam > 0:
        return 0
    u = uniform(counter_words(seed, pixel, frame)[2])
    return int(poisson_inverse_cdf(np.array([u]), lam)[0])


def gaussian(seed: int, pixel: int, frame: int) -> float:
    """N(0, 1) of one pixel: Box-Muller on block 0 words 0 and 1."""
    w = counter_words(seed, pixel, frame)
    return math.sqrt(-2.0 * math.log(uniform(w[0]))) * math.cos(2.0 * math.pi * uniform(w[1]))


def photons_per_frame(cfg) -> float:
    """Photons reaching the sensor per frame from a star of the configuration's
    magnitude: zero point x 10^(-0.4 m) x collecting area (pi/4) D^2 (1 - obs^2) x
    bandwidth x quantum efficiency x exposure dt (Table 1 wfs_source.magnitude,
    detector.bandw, detector.quantum_eff; the zero point is a parameter, the paper
    gives none). 0 for a noiseless configuration (no magnitude)."""
    if cfg.magnitude is None:
        return 0.0
    collecting_area = 0.25 * math.pi * cfg.D * cfg.D * (1.0 - cfg.obs * cfg.obs)
    flux = cfg.zero_point_ph_s_m2_nm * 10.0 ** (-0.4 * cfg.magnitude)
    return flux * collecting_area * cfg.bandwidth_nm * cfg.qe * cfg.dt_s


def apply_noise(frame_in: np.ndarray, photons_per_frame: float, n_pupil_px: int,
                read_noise_e: float, seed: int, frame_index: int) -> np.ndarray:
    """Detector frame in photo-electrons (pixels in row-major order): Poisson photon
    counts plus read noise; with photons_per_frame <= 0 the frame is returned as is."""
    flat = np.asarray(frame_in, dtype=np.float64).ravel()
    if not photons_per_frame > 0:
        return np.array(frame_in, dtype=np.float64)
    lam = flat * (photons_per_frame / n_pupil_px)
    words = [counter_words(seed, p, frame_index) for p in range(flat.size)]
    u = np.array([uniform(w[2]) for w in words])
    counts = np.zeros(flat.size)
    lit = lam > 0
    if lit.any():
        counts[lit] = poisson_inverse_cdf(u[lit], lam[lit])
    out = counts
    if read_noise_e > 0:
        g = np.array([math.sqrt(-2.0 * math.log(uniform(w[0]))) * math.cos(2.0 * math.pi * uniform(w[1]))
                      for w in words])
        out = counts + read_noise_e * g
    return out.reshape(np.shape(frame_in))
