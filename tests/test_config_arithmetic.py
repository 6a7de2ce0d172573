"""Pins of the wind displacement and the photon flux, computed by hand.

The oracle (oracle.atmosphere.wind_velocity_px, oracle.noise.photons_per_frame)
and the product (calib.wind_shift_px, calib.detector_photons) each compute these
from the workload parameters in code of their own; the expected values below are
worked out by hand from the parameters, so that a wrong pitch, direction sign or
flux factor in either copy fails here (the parity tests could not see it if both
copies shared the mistake).
"""
import math

import numpy as np
import pytest

from synth import get_config
from synth.configs import LayerSpec, with_


def _both_velocities(cfg):
    from oracle import atmosphere as at
    from paper_1607_07624_gb300 import calib
    return np.array(at.wind_velocity_px(cfg)), calib.wind_shift_px(cfg)


def test_8m_64px_wind_is_0p08_px_per_step_along_axis_0():
    # 10 m/s x 1 ms = 1 cm per step; pitch 8 m / 64 = 0.125 m; 0.01 / 0.125 = 0.08
    cfg = get_config("scao_8m_64px")
    for v in _both_velocities(cfg):
        assert v.shape == (1, 2)
        assert abs(v[0, 0] - 0.08) < 1e-15 and abs(v[0, 1]) < 1e-15


def test_elt_second_layer_splits_by_cos_and_sin_of_60_degrees():
    # layer 2 of the ELT profile: 10 m/s towards 60 degrees; pitch 39 / 480 = 0.08125 m
    # -> 0.01 / 0.08125 = 0.123076923... px per step, times (1/2, sqrt(3)/2)
    cfg = get_config("scao_elt_480px")
    d = 0.01 / 0.08125
    expect = np.array([d * 0.5, d * math.sqrt(3.0) / 2.0])
    for v in _both_velocities(cfg):
        assert v.shape == (6, 2)
        assert np.max(np.abs(v[1] - expect)) < 1e-14
        # layer 4: 25 m/s towards 180 degrees: -0.3076923... px along axis 0
        assert abs(v[3, 0] + 0.025 / 0.08125) < 1e-14 and abs(v[3, 1]) < 1e-14


def test_wind_direction_is_counter_clockwise_from_axis_0():
    cfg = with_(get_config("scao_8m_64px"), layers=(LayerSpec(1.0, 0.0, 10.0, 90.0),))
    for v in _both_velocities(cfg):
        assert abs(v[0, 0]) < 1e-15 and abs(v[0, 1] - 0.08) < 1e-15


def test_lbt_photons_per_frame_at_magnitude_10():
    # F0 = 1e8 ph / s / m^2 / nm; 10^(-0.4 x 10) = 1e-4; area (pi / 4) 8.4^2 (1 - 0.01)
    # = 54.8635 m^2; x 300 nm x 0.32 x 1e-3 s:
    # 1e8 x 1e-4 x 54.8635 x 300 x 0.32 x 1e-3 = 52 669.0 photons per frame
    from oracle import noise as nz
    from paper_1607_07624_gb300 import calib
    cfg = get_config("scao_lbt_240px")
    area = math.pi / 4.0 * 8.4 ** 2 * 0.99
    assert abs(area - 54.8635) < 1e-4
    expect = 1e4 * area * 96.0 * 1e-3
    assert abs(expect - 52669.0) < 0.1
    for photons in (nz.photons_per_frame(cfg), calib.detector_photons(cfg)):
        assert abs(photons - expect) < 1e-9 * expect


@pytest.mark.parametrize("name", ["scao_8m_64px", "scao_elt_480px"])
def test_noiseless_workloads_have_no_photons(name):
    from oracle import noise as nz
    from paper_1607_07624_gb300 import calib
    cfg = get_config(name)
    assert nz.photons_per_frame(cfg) == 0.0 and calib.detector_photons(cfg) == 0.0


def test_one_magnitude_is_a_factor_of_ten_to_the_0p4():
    from oracle import noise as nz
    from paper_1607_07624_gb300 import calib
    a, b = get_config("scao_lbt_240px"), with_(get_config("scao_lbt_240px"), magnitude=11.0)
    for f in (nz.photons_per_frame, calib.detector_photons):
        assert abs(f(a) / f(b) - 10 ** 0.4) < 1e-12
