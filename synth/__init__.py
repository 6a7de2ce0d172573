"""Seeded synthetic inputs and workload definitions.

This package is shared by the FP64 oracle, the tests and the GPU product path.
It holds workload sizes and seeded random draws only: none of the adaptive-optics
arithmetic (optics, atmosphere statistics, reconstruction) lives here.
"""
from .configs import CONFIGS, SCAOConfig, LayerSpec, get_config, tiny_config  # noqa: F401
from . import inputs  # noqa: F401
