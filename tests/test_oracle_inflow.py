"""Pins of the oracle's time-interpolated inflow series (the LES side of the
mesoscale coupling, Sec. 4): piecewise-linear interpolation in t = step * dt
reproduces linear-in-time profiles exactly, holds the end profiles outside
the series, hits every node, and with a one-profile series equals the fixed
inflow."""

import numpy as np
import pytest

from oracle.oracle import Oracle, A_U
from paper_1504_02264_gb300 import scene


def box(turb=0.0):
    return scene.box_scene(12, 8, 6, dz=scene.stretched_dz(6), turb=turb, seed=3, fixed_sweeps=1, max_sweeps=5)


def test_linear_in_time_is_exact():
    sc = box()
    o = Oracle(sc)
    z = scene.centre_heights(sc.dz)
    a, b = 1.0 + 0.1 * z, 0.05 * np.sqrt(z)
    times = np.array([0.0, 0.2, 0.7, 1.0, 2.5])
    o.set_inflow_series(times, [a + b * t for t in times])
    for s in (0, 1, 3, 5, 7, 13, 19, 20, 33, 49):
        o.step_index = s
        t = s * sc.dt
        np.testing.assert_allclose(o.inflow_profile(), a + b * t, rtol=1e-14, atol=1e-14)


def test_nodes_and_clamping():
    sc = box()
    o = Oracle(sc)
    rng = np.random.default_rng(0)
    times = np.array([0.1, 0.3, 0.6])
    prof = rng.uniform(1, 3, (3, sc.nz))
    o.set_inflow_series(times, prof)
    # steps 0-2 (t <= 0.1) and 12, 100 (t >= 0.6) are held exactly; step 6 is the
    # node t = 0.3 up to the rounding of 6 * 0.05
    for s, want in ((0, prof[0]), (1, prof[0]), (2, prof[0]), (12, prof[2]), (100, prof[2])):
        o.step_index = s
        np.testing.assert_array_equal(o.inflow_profile(), want)
    o.step_index = 6
    np.testing.assert_allclose(o.inflow_profile(), prof[1], rtol=1e-14)
    o.step_index = 9                      # t = 0.45: halfway between 0.3 and 0.6
    np.testing.assert_allclose(o.inflow_profile(), 0.5 * (prof[1] + prof[2]), rtol=1e-14)


def test_ghost_face_follows_the_series():
    sc = box()
    o = Oracle(sc)
    times = np.array([0.0, 1.0])
    prof = np.stack([np.full(sc.nz, 2.0), np.full(sc.nz, 4.0)])
    o.set_inflow_series(times, prof)
    o.step_index = 10                     # t = 0.5
    o.bc_fill()
    u = o.get(A_U)                        # (nz, ny, nx+1), face 0 = inflow plane
    np.testing.assert_allclose(u[:, :, 0], 3.0, rtol=1e-15)


def test_single_profile_series_equals_fixed_inflow():
    sc = box(turb=0.1)
    ref = Oracle(sc)
    ref.step(2)
    o = Oracle(sc)
    o.set_inflow_series([0.0], [sc.inflow_u])
    o.step(2)
    for a, b in zip(o.fields(), ref.fields()):
        assert np.array_equal(a, b)
    o.set_inflow_series([], np.zeros((0, sc.nz)))     # back to the fixed profile
    o.step(1)
    ref.step(1)
    assert np.array_equal(o.fields()[0], ref.fields()[0])


def test_times_must_increase():
    o = Oracle(box())
    with pytest.raises(ValueError):
        o.set_inflow_series([0.0, 0.0], np.ones((2, 6)))
