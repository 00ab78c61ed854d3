"""Pins of the oracle's projection (velnw) and inflow boundary (bondv1)."""

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as orc
from oracle.oracle import Oracle, A_P, A_RHS, A_U, A_V, A_W
from paper_1504_02264_gb300 import scene


def small_city(**kw):
    nx, ny, nz = 32, 24, 12
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:5, 6:12, 8:14] = 1
    solid[:3, 14:20, 18:22] = 1
    return scene.box_scene(nx, ny, nz, dz=scene.stretched_dz(nz), solid=solid, **kw)


def test_divergence_equals_dt_times_residual():
    """After velnw, div(u^{n+1}) = dt (rhs - A p + mean) cell by cell (any sweep count)."""
    sc = small_city(fixed_sweeps=1, max_sweeps=7)
    o = Oracle(sc)
    o.step(2)
    rhs = o.get(A_RHS)
    p = o.get(A_P)
    mean = o.stats()["rhs_mean"]
    fluid = sc.solid == 0
    expect = sc.dt * (rhs - o.apply_A(p) + mean) * fluid
    div = o.divergence()
    np.testing.assert_allclose(div, expect, rtol=0, atol=1e-11 * np.abs(div).max())
    assert np.abs(div).max() > 1e-4        # really not converged at 7 sweeps


def test_converged_projection_is_divergence_free():
    sc = small_city(fixed_sweeps=0, tol=1e-13, max_sweeps=100000, check_every=10)
    o = Oracle(sc)
    o.step(2)
    assert o.stats()["status"] == 0
    assert np.abs(o.divergence()).max() <= 1e-10


def test_closed_faces_exactly_zero():
    sc = small_city(fixed_sweeps=1, max_sweeps=10)
    o = Oracle(sc)
    o.step(2)
    u, v, w, _ = o.fields()
    s = sc.solid.astype(bool)
    # a face touching a building cell on either side is closed
    assert np.all(u[:, :, 1:sc.nx][s[:, :, 1:] | s[:, :, :-1]] == 0.0)
    assert np.all(v[:, 1:sc.ny, :][s[:, 1:, :] | s[:, :-1, :]] == 0.0)
    assert np.all(w[1:sc.nz][s[1:] | s[:-1]] == 0.0)
    assert np.all(w[0] == 0.0) and np.all(w[-1] == 0.0)     # ground and lid
    assert np.all(v[:, 0] == 0.0) and np.all(v[:, -1] == 0.0)  # free-slip walls


def test_laminar_inflow_face_is_the_profile():
    sc = small_city(fixed_sweeps=1, max_sweeps=3)
    o = Oracle(sc)
    o.step(1)
    u = o.get(A_U)
    np.testing.assert_array_equal(u[:, :, 0], np.broadcast_to(sc.inflow_u[:, None], u[:, :, 0].shape))


def test_splitmix64_counter_form_is_the_sequential_generator():
    """splitmix64 (Steele, Lea & Flood 2014): state += 0x9E3779B97F4A7C15, output
    = mix(state).  The counter form used for the inflow must give the ctr-th output."""
    M = (1 << 64) - 1

    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    seed = 0x1234ABCD
    state = seed
    for ctr in range(64):
        state = (state + 0x9E3779B97F4A7C15) & M
        assert orc.splitmix64(seed, ctr) == mix(state)


def test_box_muller_is_standard_normal():
    x = np.array([orc.gauss(7, c) for c in range(20000)])
    assert abs(x.mean()) < 0.03 and abs(x.std() - 1.0) < 0.03
    assert stats.kstest(x, "norm").pvalue > 1e-3


def test_turbulent_inflow_intensity():
    sc = small_city(fixed_sweeps=1, max_sweeps=2, turb=0.1, seed=5)
    o = Oracle(sc)
    o.bc_fill()
    uin = o.raw(A_U)[1:sc.nz + 1, 1:sc.ny + 1, 0]
    U = sc.inflow_u[:, None]
    rel = (uin / U - 1.0)[U[:, 0] > 0]
    assert abs(rel.std() - 0.1) < 0.02
    assert abs(rel.mean()) < 0.02
