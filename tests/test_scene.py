"""The seeded synthetic inputs match the workload recipe they stand for: grid
sizes, stretched spacing, log-law inflow, building counts, footprints, plan
density, heights and the clear inflow/outflow margins (the generator holds no
method arithmetic; these tests check its own contract)."""
import numpy as np
import pytest
import scipy.ndimage as ndi

from paper_1504_02264_gb300 import scene


def _tops(sc, lab, n):
    """Height of the top face of each labelled building's column (m)."""
    zt = np.cumsum(sc.dz)
    out = []
    for b in range(1, n + 1):
        col = sc.solid[:, lab == b][:, 0]
        out.append(zt[np.nonzero(col)[0].max()])
    return np.array(out)


def test_stretched_spacing_and_log_law():
    dz = scene.stretched_dz(32)
    assert dz[0] == pytest.approx(2.0) and dz[-1] == pytest.approx(8.0)
    np.testing.assert_allclose(dz[1:] / dz[:-1], (8.0 / 2.0) ** (1 / 31), rtol=1e-12)
    z = np.array([0.05, 0.1, 1.0, 10.0])
    u = scene.log_law(z, 0.3, 0.1)
    assert u[0] == 0.0 and u[1] == 0.0
    assert u[3] == pytest.approx(0.3 / scene.KAPPA * np.log(100.0))


def test_lattice_workload():
    sc = scene.lattice_scene(0)
    assert (sc.nx, sc.ny, sc.nz) == (64, 64, 32)
    lab, n = ndi.label(sc.solid[0] > 0)
    assert n == 16
    assert all(int((lab == b).sum()) == 64 for b in range(1, n + 1))       # 8 x 8 footprints
    tops = _tops(sc, lab, n)
    assert tops.min() >= 10.0 - 8.0 and tops.max() <= 40.0 + 8.0           # U(10, 40) m, level-quantised
    assert sc.fixed_sweeps == 1 and sc.max_sweeps == 50


@pytest.mark.parametrize("seed", [0, 1])
def test_random_city_workload(seed):
    sc = scene.random_scene(seed)
    assert (sc.nx, sc.ny, sc.nz) == (150, 150, 90)
    foot = sc.solid[0] > 0
    lab, n = ndi.label(foot)
    assert n == 100                                          # 100 separate cuboids (1-cell gaps)
    assert 0.29 <= foot.mean() <= 0.31                       # 30% plan density
    assert sc.solid[:, :, :16].sum() == 0 and sc.solid[:, :, -16:].sum() == 0
    assert 14.0 <= np.median(_tops(sc, lab, n)) <= 26.0     # lognormal heights, median 20 m
    np.testing.assert_array_equal(sc.inflow_u, scene.log_law(scene.centre_heights(sc.dz), 0.3, 0.1))
    assert sc.turb == pytest.approx(0.1) and sc.tol == pytest.approx(1e-6)


def test_ensemble_workload():
    es = scene.ensemble_scenes(0)
    assert len(es) == 32
    k = scene.KAPPA
    for sc in es:
        assert 96 <= sc.nx <= 256 and 96 <= sc.ny <= 256 and 64 <= sc.nz <= 128
        z, U = scene.centre_heights(sc.dz), sc.inflow_u
        i1, i2 = 10, 40                                        # two heights above every z0
        ustar = k * (U[i2] - U[i1]) / np.log(z[i2] / z[i1])
        z0 = z[i1] * np.exp(-k * U[i1] / ustar)
        assert 0.2 <= ustar <= 0.6 and 0.05 <= z0 <= 0.5        # the member's own log-law inflow
    assert len({(sc.nx, sc.ny, sc.nz) for sc in es}) > 16       # uneven sizes
