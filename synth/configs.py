"""Workload definitions for the single-conjugate pyramid AO loop.

The parameter names follow the paper's parameter file (Table 1: main, DM, pyramid,
detector, wfs_source, atmo, seeing, wind_speed, wind_direction, control). The sizes
are the synthetic workloads this project measures on; every number is written out
here so that the oracle and the GPU path read the same values and neither derives
them from the other.

Conventions shared by both sides (readings of the paper, which gives no formulas):
  * array axis 0 is x (rows), axis 1 is y (columns);
  * OPD in nm, phase = 2*pi*OPD/lambda;
  * wind direction counter-clockwise from axis 0.

The arithmetic of the method (wind displacement per step, photon flux) is not
here: the oracle and the product each compute it from these parameters.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Tuple


@dataclass(frozen=True)
class LayerSpec:
    fraction: float          # Cn2 weight (the weights of one atmosphere sum to 1)
    height_m: float          # layer altitude [m]; on-axis source: no footprint scaling
    wind_mps: float          # wind speed [m/s]
    wind_dir_deg: float = 0.0  # counter-clockwise from array axis 0


@dataclass(frozen=True)
class SCAOConfig:
    name: str
    D: float                 # telescope diameter [m]
    Np: int                  # pupil pixels across
    N: int                   # FFT grid (focal/pupil plane) size
    obs: float               # central obstruction ratio
    n_sub: int               # sub-apertures across
    K: int                   # modulation points
    mod_radius: float        # modulation radius [lambda/D]
    wavelength_nm: float     # pyramid wavelength
    n_modes: int             # DM modes
    basis: str               # 'zernike' (Noll j = 2 ..) or 'kl'
    r0_m: float              # Fried parameter at 500 nm [m]
    L0_m: float              # outer scale [m]
    layers: Tuple[LayerSpec, ...]
    S: int                   # phase-screen size (periodic, pitch = D/Np)
    n_steps: int             # simulated loop steps
    dt_s: float = 1e-3       # loop step [s]
    gain: float = 0.5        # integrator gain, all modes
    delay: int = 1           # measurement at step t sees the command of step t-delay
    pushpull_nm: float = 10.0  # interaction-matrix push-pull amplitude [nm RMS]
    magnitude: float | None = None     # None: noiseless
    read_noise_e: float = 0.0
    bandwidth_nm: float = 300.0        # detector bandwidth (Table 1 example)
    qe: float = 0.32                   # quantum efficiency x transmission (Table 1 example)
    zero_point_ph_s_m2_nm: float = 1.0e8   # photon zero point (the paper gives none)
    seed: int = 1000

    # ---- simple bookkeeping (sizes only) ----
    @property
    def dx(self) -> float:
        return self.D / self.Np

    @property
    def b(self) -> int:
        """Detector binning factor (fine pixels per sub-aperture side)."""
        assert self.N % (2 * self.n_sub) == 0
        return self.N // (2 * self.n_sub)

    @property
    def n_det(self) -> int:
        return 2 * self.n_sub

    @property
    def delta(self) -> float:
        """Pyramid face phase slope: pupil images centred in the grid quadrants."""
        return self.N / 4.0


CFG1 = SCAOConfig(
    name="scao_8m_64px", D=8.0, Np=64, N=128, obs=0.1, n_sub=16, K=12, mod_radius=3.0,
    wavelength_nm=750.0, n_modes=100, basis="zernike", r0_m=0.15, L0_m=25.0,
    layers=(LayerSpec(1.0, 0.0, 10.0, 0.0),), S=1024, n_steps=200, seed=1000)

CFG2 = SCAOConfig(
    name="scao_lbt_240px", D=8.4, Np=240, N=480, obs=0.1, n_sub=30, K=24, mod_radius=3.0,
    wavelength_nm=750.0, n_modes=400, basis="kl", r0_m=0.12, L0_m=25.0,
    layers=(LayerSpec(0.60, 0.0, 8.0, 0.0), LayerSpec(0.25, 4000.0, 15.0, 0.0),
            LayerSpec(0.15, 10000.0, 25.0, 0.0)),
    S=4096, n_steps=2000, magnitude=10.0, read_noise_e=0.5, seed=1000)

CFG3 = SCAOConfig(
    name="scao_elt_480px", D=39.0, Np=480, N=960, obs=0.1, n_sub=96, K=32, mod_radius=4.0,
    wavelength_nm=750.0, n_modes=4000, basis="kl", r0_m=0.10, L0_m=25.0,
    layers=(LayerSpec(0.45, 0.0, 6.0, 0.0), LayerSpec(0.15, 1000.0, 10.0, 60.0),
            LayerSpec(0.12, 3000.0, 15.0, 120.0), LayerSpec(0.10, 6000.0, 25.0, 180.0),
            LayerSpec(0.10, 10000.0, 20.0, 240.0), LayerSpec(0.08, 15000.0, 12.0, 300.0)),
    S=2048, n_steps=1000, seed=1000)

CONFIGS = {c.name: c for c in (CFG1, CFG2, CFG3)}

# Batched Monte-Carlo workload: loops of three sizes stepped together. Per group
# (count, configuration): 8 m / 128 px / 20x20 sub-apertures / 12 points, 25 m /
# 320 px / 60x60 / 24, 39 m / 480 px / 96x96 / 32. Not stated for this workload and
# taken here: one von Karman layer per loop (10 m/s), modulation 3 lambda/D, about
# half as many modes as valid sub-apertures, 1 ms steps, noiseless.
BATCH_GROUPS = (
    (32, SCAOConfig(name="batch_8m_128px", D=8.0, Np=128, N=256, obs=0.1, n_sub=20, K=12, mod_radius=3.0,
                    wavelength_nm=750.0, n_modes=150, basis="zernike", r0_m=0.15, L0_m=25.0,
                    layers=(LayerSpec(1.0, 0.0, 10.0, 0.0),), S=512, n_steps=200, seed=3000)),
    (24, SCAOConfig(name="batch_25m_320px", D=25.0, Np=320, N=640, obs=0.1, n_sub=60, K=24, mod_radius=3.0,
                    wavelength_nm=750.0, n_modes=1400, basis="zernike", r0_m=0.15, L0_m=25.0,
                    layers=(LayerSpec(1.0, 0.0, 10.0, 0.0),), S=1024, n_steps=200, seed=4000)),
    (8, SCAOConfig(name="batch_39m_480px", D=39.0, Np=480, N=960, obs=0.1, n_sub=96, K=32, mod_radius=3.0,
                   wavelength_nm=750.0, n_modes=3578, basis="zernike", r0_m=0.15, L0_m=25.0,
                   layers=(LayerSpec(1.0, 0.0, 10.0, 0.0),), S=2048, n_steps=200, seed=5000)),
)


def batched_workload(r0_range=(0.08, 0.2), seed: int = 9000):
    """The 64 loops of the batched workload: [(group index, configuration)] with a
    seed and an r0 (uniform in r0_range) of their own."""
    from .inputs import rng
    g = rng(seed)
    out = []
    for gi, (count, cfg) in enumerate(BATCH_GROUPS):
        for i in range(count):
            out.append((gi, with_(cfg, seed=cfg.seed + 17 * i, r0_m=float(g.uniform(*r0_range)))))
    return out


def get_config(name: str) -> SCAOConfig:
    """A workload by name: scao_8m_64px, scao_lbt_240px or scao_elt_480px."""
    return CONFIGS[name]


def tiny_config(Np: int = 16, N: int | None = None, n_sub: int = 4, K: int = 4,
                mod_radius: float = 2.0, n_modes: int = 10, **kw) -> SCAOConfig:
    """Small systems for exhaustive tests (brute-force sizes)."""
    N = 2 * Np if N is None else N
    base = dict(name=f"tiny_{Np}px", D=Np * 0.125, Np=Np, N=N, obs=0.1, n_sub=n_sub, K=K,
                mod_radius=mod_radius, wavelength_nm=750.0, n_modes=n_modes,
                basis="zernike", r0_m=0.15, L0_m=25.0,
                layers=(LayerSpec(1.0, 0.0, 10.0, 0.0),), S=64, n_steps=20, seed=7)
    base.update(kw)
    return SCAOConfig(**base)


def with_(cfg: SCAOConfig, **kw) -> SCAOConfig:
    return replace(cfg, **kw)
