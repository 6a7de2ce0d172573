"""Pins of the oracle's extended-source pyramid (oracle/optics.pwfs_intensity_extended)
against what the optics fixes: a one-point source is the point source, an offset
point seen unmodulated is the modulated point source on that offset, a ring of points
is the modulation circle, the axes swap under transposition, and the pure-phase mask
with unitary transforms conserves the pupil's flux for any source."""
import math

import numpy as np

from oracle import optics as op

LAM, Np, N = 750.0, 16, 32


def _opd(seed):
    return np.random.default_rng(seed).standard_normal((Np, Np)) * 80.0


def test_one_point_at_the_origin_is_the_point_source():
    opd = _opd(1)
    a = op.pwfs_intensity_extended(opd, LAM, 0.1, N, 8, 2.0, [0.0], [0.0])
    b = op.pwfs_intensity(opd, LAM, 0.1, N, 8, 2.0)
    assert np.array_equal(a, b)


def test_offset_point_unmodulated_is_the_one_point_modulation():
    """theta_0 = 0: one modulation point of radius r tilts by (r, 0), the same as a
    source point at (+r, 0); a point at (-r, 0) is not (the sign is fixed)."""
    opd = _opd(2)
    r = 1.75
    a = op.pwfs_intensity_extended(opd, LAM, 0.1, N, 1, 0.0, [r], [0.0])
    b = op.pwfs_intensity(opd, LAM, 0.1, N, 1, r)
    assert np.max(np.abs(a - b)) < 1e-10 * b.max()
    c = op.pwfs_intensity_extended(opd, LAM, 0.1, N, 1, 0.0, [-r], [0.0])
    assert np.max(np.abs(c - b)) > 1e-3 * b.max()


def test_ring_of_points_is_the_modulation_circle():
    opd = _opd(3)
    K, r = 12, 2.5
    th = 2 * np.pi * np.arange(K) / K
    a = op.pwfs_intensity_extended(opd, LAM, 0.0, N, 1, 0.0, r * np.cos(th), r * np.sin(th))
    b = op.pwfs_intensity(opd, LAM, 0.0, N, K, r)
    assert np.max(np.abs(a - b)) < 1e-10 * b.max()


def test_transposition_swaps_the_source_axes():
    """The pupil and the mask are symmetric under swapping the axes, so transposing
    the wavefront and swapping (ex, ey) transposes the image (K a multiple of 4: the
    modulation circle maps onto itself, theta -> pi/2 - theta); with an asymmetric
    source this fixes the y offset's sign against x's."""
    opd = _opd(4)
    ex, ey, w = [0.0, 1.5, -0.5], [0.7, -1.0, 2.0], [1.0, 2.0, 0.5]
    a = op.pwfs_intensity_extended(opd, LAM, 0.1, N, 8, 1.5, ex, ey, w)
    b = op.pwfs_intensity_extended(opd.T, LAM, 0.1, N, 8, 1.5, ey, ex, w)
    assert np.max(np.abs(a - b.T)) < 1e-10 * a.max()
    c = op.pwfs_intensity_extended(opd.T, LAM, 0.1, N, 8, 1.5, ey, [-x for x in ex], w)
    assert np.max(np.abs(a - c.T)) > 1e-3 * a.max()


def test_flux_is_conserved_for_any_source():
    opd = _opd(5)
    A = op.pupil_mask(Np, 0.1)
    g = np.random.default_rng(6)
    I = op.pwfs_intensity_extended(opd, LAM, 0.1, N, 4, 1.0, g.uniform(-3, 3, 5), g.uniform(-3, 3, 5),
                                   g.uniform(0.1, 1.0, 5))
    assert abs(I.sum() - A.sum()) < 1e-9 * A.sum()


def test_weights_are_normalised():
    opd = _opd(7)
    a = op.pwfs_intensity_extended(opd, LAM, 0.1, N, 4, 1.0, [0.0, 1.0], [0.0, 0.0], [3.0, 1.0])
    p0 = op.pwfs_intensity_extended(opd, LAM, 0.1, N, 4, 1.0, [0.0], [0.0])
    p1 = op.pwfs_intensity_extended(opd, LAM, 0.1, N, 4, 1.0, [1.0], [0.0])
    assert np.max(np.abs(a - (0.75 * p0 + 0.25 * p1))) < 1e-12 * a.max()
