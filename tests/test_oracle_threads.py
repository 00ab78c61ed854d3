"""The OpenMP build of the oracle (used to time the CPU baseline on every
host core) against the sequential build: same source, same arithmetic, so a
two tolerance-mode steps of a city with turbulent inflow, a periodic-y city
and a twinned-buffer run must agree bit for bit, whatever the thread count."""

import numpy as np
import pytest

from oracle import oracle as orc
from oracle.oracle import Oracle, A_NUT, A_RHS
from paper_1504_02264_gb300 import scene


def city(periodic_y=False):
    rng = np.random.default_rng(5)
    nx, ny, nz = 36, 24, 12
    solid = np.zeros((nz, ny, nx), np.uint8)
    for _ in range(4):
        x0, y0, h = int(rng.integers(4, nx - 10)), int(rng.integers(1, ny - 6)), int(rng.integers(2, nz - 2))
        solid[:h, y0:y0 + 5, x0:x0 + 6] = 1
    bc = (scene.BC_INOUT, scene.BC_PERIODIC if periodic_y else scene.BC_FREESLIP, scene.BC_WALL)
    return scene.box_scene(nx, ny, nz, dz=scene.stretched_dz(nz), solid=solid, bc=bc, turb=0.1, seed=4,
                           tol=1e-6, max_sweeps=4000, check_every=10)


def run(sc, omp):
    o = Oracle(sc, omp=omp)
    stats = []
    for _ in range(2):
        o.step(1)
        stats.append(o.stats())
    return [o.get(a) for a in (A_NUT, A_RHS)] + list(o.fields()), stats


@pytest.mark.parametrize("periodic_y", [False, True])
@pytest.mark.parametrize("threads", [3, 8])
def test_openmp_build_bit_identical(periodic_y, threads):
    orc.set_threads(threads)
    assert orc.threads(True) == threads
    assert orc.threads(False) == 1
    sc = city(periodic_y)
    a, sa = run(sc, False)
    b, sb = run(sc, True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert sa == sb
    assert all(s["sweeps"] > 10 for s in sa)


def test_openmp_twinned_bit_identical():
    orc.set_threads(4)
    sc = city()
    outs = []
    for omp in (False, True):
        o = Oracle(sc, omp=omp)
        o.step(1)
        o.twin_sweeps(7, 0.9)
        outs.append(o.get(orc.A_P))
    assert np.array_equal(outs[0], outs[1])
