"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

The FP64 instantiation of the kernels must agree with the oracle to ~1e-11
(same discretisation, only rounding order differs), which separates indexing
mistakes from rounding.  The FP32 production path must keep the max relative
velocity error <= 1e-4 after 20 steps of the 64x64x32 lattice workload.
Relative error = max |gpu - oracle| / max |oracle| over the array."""

import numpy as np
import pytest

from oracle.oracle import (Oracle, A_U, A_V, A_W, A_P, A_NUT, A_RHS, A_US, A_VS, A_WS,
                           A_FU, A_FV, A_FW)
from paper_1504_02264_gb300 import scene

pytestmark = pytest.mark.gpu

les = pytest.importorskip("paper_1504_02264_gb300.les")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    les.lib()
    yield


def rel(a, b):
    scale = max(np.abs(b).max(), 1e-300)
    return float(np.abs(np.asarray(a, np.float64) - b).max() / scale)


def city(nx=40, ny=24, nz=12, turb=0.0, periodic_y=False, seed=3, **kw):
    rng = np.random.default_rng(seed)
    solid = np.zeros((nz, ny, nx), np.uint8)
    for _ in range(4):
        x0 = int(rng.integers(4, nx - 10))
        y0 = int(rng.integers(1, ny - 6))
        h = int(rng.integers(2, nz - 2))
        solid[:h, y0:y0 + 5, x0:x0 + 6] = 1
    bc = (scene.BC_INOUT, scene.BC_PERIODIC if periodic_y else scene.BC_FREESLIP, scene.BC_WALL)
    return scene.box_scene(nx, ny, nz, dz=scene.stretched_dz(nz), solid=solid, bc=bc, turb=turb,
                           seed=seed, **kw)


def compare_fields(dom, o, tol):
    errs = {}
    for name, g, r in zip("uvwp", dom.fields(), o.fields()):
        errs[name] = rel(g, r)
    assert max(errs.values()) <= tol, errs
    return errs


# ---------------------------------------------------------------------------
# FP64: discretisation parity, phase by phase and over several steps

@pytest.mark.parametrize("turb", [0.0, 0.1])
def test_fp64_phases_one_step(turb):
    sc = city(turb=turb, fixed_sweeps=1, max_sweeps=15)
    d = les.Domain(sc, precision=les.LES_FP64)
    o = Oracle(sc)
    d.step(1)
    o.step(1)
    pairs = [(les.LES_AUX_NUT, A_NUT), (les.LES_AUX_RHS, A_RHS), (les.LES_AUX_USTAR, A_US),
             (les.LES_AUX_VSTAR, A_VS), (les.LES_AUX_WSTAR, A_WS), (les.LES_AUX_FU, A_FU),
             (les.LES_AUX_FV, A_FV), (les.LES_AUX_FW, A_FW)]
    for aux, arr in pairs:
        assert rel(d.aux(aux), o.get(arr)) <= 1e-12, aux
    compare_fields(d, o, 1e-11)


@pytest.mark.parametrize("case", ["city", "city_turb", "periodic_y", "odd_sizes", "tiny", "periodic_xyz"])
def test_fp64_multi_step(case):
    if case == "city":
        sc = city(fixed_sweeps=1, max_sweeps=20)
    elif case == "city_turb":
        sc = city(turb=0.1, fixed_sweeps=1, max_sweeps=20)
    elif case == "periodic_y":
        sc = city(periodic_y=True, ny=24, turb=0.1, fixed_sweeps=1, max_sweeps=20)
    elif case == "odd_sizes":
        sc = city(nx=33, ny=17, nz=9, fixed_sweeps=1, max_sweeps=20)
    elif case == "tiny":
        sc = scene.box_scene(2, 2, 2, fixed_sweeps=1, max_sweeps=3)
    else:
        n = 16
        sc = scene.box_scene(n, n, 4, dx=0.4, dy=0.4, dz=np.full(4, 0.4),
                             bc=(scene.BC_PERIODIC,) * 3, nu=0.01, dt=0.02, fixed_sweeps=1,
                             max_sweeps=30)
        u, v, w, p = scene.random_fields(sc, 5, amp=0.3)
        u[:, :, 0] = u[:, :, -1]
        v[:, 0, :] = v[:, -1, :]
        w[0] = w[-1]
        sc.u0, sc.v0, sc.w0, sc.p0 = u, v, w, 0 * p
    d = les.Domain(sc, precision=les.LES_FP64)
    o = Oracle(sc)
    for _ in range(5):
        sd = d.step(1)
        o.step(1)
        so = o.stats()
        assert abs(sd["rel_residual"] - so["rel_residual"]) <= 1e-9 * max(1.0, so["rel_residual"])
        assert abs(sd["mass_factor"] - so["mass_factor"]) <= 1e-12
    compare_fields(d, o, 1e-11)


def test_fp64_pressure_solve_random_rhs():
    sc = city(fixed_sweeps=1, max_sweeps=60)
    rhs = scene.random_rhs(sc, 9)
    d = les.Domain(sc, precision=les.LES_FP64)
    o = Oracle(sc)
    sd = d.pressure_solve(rhs)
    o.pressure_solve(rhs)
    assert rel(d.fields()[3], o.get(A_P)) <= 1e-11
    assert abs(sd["rel_residual"] - o.stats()["rel_residual"]) <= 1e-10


def test_fp64_tolerance_mode_same_sweeps():
    sc = city(fixed_sweeps=0, tol=1e-6, max_sweeps=5000, check_every=10)
    d = les.Domain(sc, precision=les.LES_FP64)
    o = Oracle(sc)
    for _ in range(3):
        sd = d.step(1)
        o.step(1)
        assert sd["sweeps"] == o.stats()["sweeps"]
        assert sd["rc"] == 0 and sd["rel_residual"] <= 1e-6
    compare_fields(d, o, 1e-10)


# ---------------------------------------------------------------------------
# FP32 production path

def test_fp32_lattice_20_steps_parity():
    """64x64x32 lattice, 20 steps, exactly 50 sweeps per step: max relative
    velocity error against the FP64 oracle <= 1e-4."""
    sc = scene.lattice_scene(0)
    d = les.Domain(sc, precision=les.LES_FP32)
    o = Oracle(sc)
    d.step(20)
    o.step(20)
    g = d.fields()
    r = o.fields()
    vel_scale = max(np.abs(a).max() for a in r[:3])
    err = max(np.abs(np.asarray(a, np.float64) - b).max() for a, b in zip(g[:3], r[:3])) / vel_scale
    print(f"FP32 lattice 20 steps: max relative velocity error {err:.3e}")
    assert err <= 1e-4


def test_fp32_phases_and_solve():
    sc = city(turb=0.1, fixed_sweeps=1, max_sweeps=40)
    d = les.Domain(sc, precision=les.LES_FP32)
    o = Oracle(sc)
    d.step(3)
    o.step(3)
    for aux, arr in [(les.LES_AUX_NUT, A_NUT), (les.LES_AUX_USTAR, A_US), (les.LES_AUX_RHS, A_RHS)]:
        assert rel(d.aux(aux), o.get(arr)) <= 2e-4, aux
    compare_fields(d, o, 2e-4)


def test_fp32_converged_step_is_divergence_free():
    """Tolerance mode: every FP32 step reaches FP64 relative residual 1e-6, and
    the projected GPU velocity has ||div u|| <= 1e-6 ||div u*|| plus the
    rounding floor of storing the faces in FP32 (checked by the oracle)."""
    sc = city(turb=0.1, fixed_sweeps=0, tol=1e-6, max_sweeps=20000, check_every=10)
    d = les.Domain(sc, precision=les.LES_FP32)
    for _ in range(3):
        st = d.step(1)
        assert st["rc"] == 0 and st["rel_residual"] <= 1e-6, st
    star = Oracle(sc)
    star.set(A_U, d.aux(les.LES_AUX_USTAR).astype(np.float64))
    star.set(A_V, d.aux(les.LES_AUX_VSTAR).astype(np.float64))
    star.set(A_W, d.aux(les.LES_AUX_WSTAR).astype(np.float64))
    div_star = star.divergence()
    chk = Oracle(sc)
    u, v, w, p = [a.astype(np.float64) for a in d.fields()]
    chk.set_fields(u, v, w, p)
    div = chk.divergence()
    # |div| of the exact projection rounded to FP32 face values
    dz = sc.dz[:, None, None]
    mag = ((np.abs(u[:, :, 1:]) + np.abs(u[:, :, :-1])) / sc.dx + (np.abs(v[:, 1:]) + np.abs(v[:, :-1])) / sc.dy +
           (np.abs(w[1:]) + np.abs(w[:-1])) / dz) * (sc.solid == 0)
    floor = 2.0 ** -24 * np.linalg.norm(mag)
    assert np.linalg.norm(div) <= 1e-6 * np.linalg.norm(div_star) + 3 * floor


# ---------------------------------------------------------------------------
# checkpoint / restart and error paths

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_checkpoint_resume_bitwise(prec):
    p = les.LES_FP64 if prec == "fp64" else les.LES_FP32
    sc = city(turb=0.1, fixed_sweeps=0, tol=1e-5, max_sweeps=3000, check_every=10)
    a = les.Domain(sc, precision=p)
    a.step(4)
    ref = a.fields()
    b = les.Domain(sc, precision=p)
    b.step(2)
    blob = b.get_state()
    c = les.Domain(sc, precision=p)
    c.set_state(blob)
    c.step(2)
    for x, y in zip(ref, c.fields()):
        assert np.array_equal(x, y)


def test_set_state_rejects_other_grid():
    a = les.Domain(city(), precision=les.LES_FP32)
    b = les.Domain(city(nx=42), precision=les.LES_FP32)
    with pytest.raises(les.LesError) as e:
        b.set_state(a.get_state())
    assert e.value.code == les.LES_ESTATE


def test_no_convergence_status():
    sc = city(fixed_sweeps=0, tol=1e-14, max_sweeps=20, check_every=10)
    d = les.Domain(sc, precision=les.LES_FP32)
    st = d.step(1)
    assert st["rc"] == les.LES_ENOCONV and st["sweeps"] == 20


# ---------------------------------------------------------------------------
# fused red-black kernel: every tile shape / k-chunk gives the two-pass iterate

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("case", ["city", "periodic_y_odd", "periodic_xyz"])
def test_fused_sor_matches_two_pass(prec, case):
    p = les.LES_FP64 if prec == "fp64" else les.LES_FP32
    if case == "city":
        sc = city(nx=37, ny=21, nz=11, turb=0.1, fixed_sweeps=1, max_sweeps=17)
    elif case == "periodic_y_odd":
        sc = city(nx=45, ny=18, nz=13, periodic_y=True, turb=0.1, fixed_sweeps=1, max_sweeps=9)
    else:
        n = 12
        sc = scene.box_scene(n, n, 6, dx=0.4, dy=0.4, dz=np.full(6, 0.4), bc=(scene.BC_PERIODIC,) * 3,
                             nu=0.01, dt=0.02, fixed_sweeps=1, max_sweeps=11)
        u, v, w, q = scene.random_fields(sc, 6, amp=0.3)
        u[:, :, 0] = u[:, :, -1]
        v[:, 0, :] = v[:, -1, :]
        w[0] = w[-1]
        sc.u0, sc.v0, sc.w0, sc.p0 = u, v, w, 0 * q
    ref = les.Domain(sc, precision=p)
    ref.set_sor_config(-1, 0)
    ref.step(2)
    want = ref.fields()
    tol = 0.0 if prec == "fp64" else 1e-6
    # TMA block tiles (17-20), k-marching TMA columns (25-28) and column-walk
    # TMA blocks (29-34) on every FP32 grid, periodic halos
    # included; the persistent TMA tiles (21-24) only without periodic axes
    tiles = list(range(17))
    if prec == "fp32":
        tiles += list(range(17, 21)) + (list(range(21, 25)) if case == "city" else []) + list(range(25, 35))
    if prec == "fp32" and case != "city":
        d = les.Domain(sc, precision=p)
        for tile in range(21, 25):
            with pytest.raises(les.LesError):
                d.set_sor_config(tile, 0)
        d.close()
    for tile in tiles:
        for kc in ((0, 3, 5) if (tile < 6 or 25 <= tile < 29) else (0,)):
            d = les.Domain(sc, precision=p)
            d.set_sor_config(tile, kc)
            d.step(2)
            for a, b in zip(d.fields(), want):
                scale = max(np.abs(b).max(), 1e-30)
                assert np.abs(a.astype(np.float64) - b).max() <= tol * scale, (tile, kc)
            d.close()


@pytest.mark.parametrize("case", ["city", "periodic_y_odd"])
def test_column_walk_equals_masked_update(case):
    """The column-walk TMA blocks (tiles 29-34) drop the open-face masks of
    the neighbour coefficients (a closed face meets a cell whose correction
    is zero) and keep the masked update's products and sums in the same
    order: after several steps of sweeps to tolerance the fields equal those
    of the masked TMA block kernel (tile 17) bit for bit."""
    if case == "city":
        sc = city(nx=61, ny=37, nz=19, turb=0.1, fixed_sweeps=0, tol=1e-6, max_sweeps=4000, check_every=10)
    else:
        sc = city(nx=45, ny=18, nz=13, periodic_y=True, turb=0.1, fixed_sweeps=0, tol=1e-6, max_sweeps=4000,
                  check_every=10)
    out = {}
    for tile in (17, 29, 30, 31, 32, 33, 34):
        d = les.Domain(sc, precision=les.LES_FP32)
        d.set_sor_config(tile, 0)
        sweeps = [d.step(1)["sweeps"] for _ in range(3)]
        out[tile] = (sweeps, d.fields())
        d.close()
    for tile in (29, 30, 31, 32, 33, 34):
        assert out[tile][0] == out[17][0], tile
        for a, b in zip(out[tile][1], out[17][1]):
            assert np.array_equal(a, b), tile


def test_autotune_picks_a_valid_config():
    sc = city(nx=64, ny=48, nz=24, fixed_sweeps=1, max_sweeps=10)
    d = les.Domain(sc, precision=les.LES_FP32)
    d.step(1)
    (tile, kc), ms = d.autotune_sor(sweeps=5)
    assert 0 <= tile < les.LES_SOR_NTILES and ms > 0
    before = d.fields()
    d2 = les.Domain(sc, precision=les.LES_FP32)
    d2.step(1)
    for a, b in zip(before, d2.fields()):
        assert np.array_equal(a, b)      # tuning sweeps never touch the state


# ---------------------------------------------------------------------------
# CUDA-graph step (device-side stop test) against the host-driven loop

@pytest.mark.parametrize("mode", ["tol", "tol_remainder", "fixed"])
def test_graph_step_matches_host_loop(mode):
    if mode == "tol":
        sc = city(turb=0.1, fixed_sweeps=0, tol=1e-6, max_sweeps=5000, check_every=10)
    elif mode == "tol_remainder":
        sc = city(turb=0.1, fixed_sweeps=0, tol=1e-12, max_sweeps=37, check_every=10)
    else:
        sc = city(turb=0.1, fixed_sweeps=1, max_sweeps=23)
    a = les.Domain(sc, precision=les.LES_FP64)
    a.set_graph(False)
    b = les.Domain(sc, precision=les.LES_FP64)
    b.set_graph(True)
    for _ in range(3):
        sa = a.step(1)
        sb = b.step(1)
        # a sweep budget that is not a whole number of batches runs the host loop
        assert sb["graph"] == (0 if mode == "tol_remainder" else 1) and sa["graph"] == 0
        assert sa["sweeps"] == sb["sweeps"] and sa["rc"] == sb["rc"], (sa, sb)
        assert sa["step"] == sb["step"]
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    if mode == "tol_remainder":
        assert sb["rc"] == les.LES_ENOCONV and sb["sweeps"] == 37


def test_graph_multi_step_call_matches_single_steps():
    sc = city(turb=0.1, fixed_sweeps=0, tol=1e-6, max_sweeps=5000, check_every=10)
    a = les.Domain(sc, precision=les.LES_FP32)
    for _ in range(4):
        a.step(1)
    b = les.Domain(sc, precision=les.LES_FP32)
    st = b.step(4)
    assert st["step"] == 4 and st["rc"] == 0
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)


def test_fp64_inflow_series_matches_oracle():
    """A time-varying inflow series (interpolated in time, turbulence on top)
    gives the oracle's step to FP64 rounding over several steps."""
    sc = city(turb=0.1)
    z = scene.centre_heights(sc.dz)
    times = np.array([0.0, 0.08, 0.2, 0.3])
    prof = np.stack([sc.inflow_u * (1.0 + 0.3 * np.sin(3.0 * t)) + 0.01 * t * z for t in times])
    o = Oracle(sc)
    o.set_inflow_series(times, prof)
    d = les.Domain(sc, precision=les.LES_FP64)
    d.set_inflow_series(times, prof)
    o.step(6)
    d.step(6)
    compare_fields(d, o, 1e-11)
    d.close()


# ---------------------------------------------------------------------------
# les_sor_compare: the solver's red-black SOR and the paper's twinned double
# buffer (Sec. 2.6) on one pressure problem, against the oracle

def _compatible_problem(sc, seed):
    rng = np.random.default_rng(seed)
    fluid = sc.solid == 0
    rhs = rng.standard_normal(sc.solid.shape) * fluid
    w = np.broadcast_to(sc.dz[:, None, None], rhs.shape)[fluid]
    rhs[fluid] -= np.sum(w * rhs[fluid]) / np.sum(w)
    p0 = rng.standard_normal(sc.solid.shape) * fluid
    return rhs, p0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("variant", ["redblack", "twinned"])
def test_sor_compare_matches_oracle(prec, variant):
    sc = city(nx=40, ny=24, nz=12, periodic_y=True, fixed_sweeps=1, max_sweeps=10)
    rhs, p0 = _compatible_problem(sc, 21)
    sweeps = 7
    o = Oracle(sc)
    o.set(A_P, p0)
    o.set(A_RHS, rhs)
    if variant == "twinned":
        omega, vid = 0.9, les.LES_SOR_TWINNED
        o.twin_sweeps(sweeps, omega)
    else:
        omega, vid = -1.0, les.LES_SOR_REDBLACK      # the grid's 1.7, as in the oracle
        o.sor_sweeps(sweeps)
    want = o.get(A_P)
    want_rel = o.residual()
    d = les.Domain(sc, precision=les.LES_FP64 if prec == "fp64" else les.LES_FP32)
    d.step(1)
    before = d.fields()
    got, ms, rel = d.sor_compare(vid, omega, sweeps, rhs, p0)
    after = d.fields()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)                  # the handle's state is untouched
    scale = np.abs(want).max()
    tol = 1e-11 if prec == "fp64" else 1e-5
    assert np.abs(got - want).max() <= tol * scale, (np.abs(got - want).max(), scale)
    assert rel == pytest.approx(want_rel, rel=1e-9 if prec == "fp64" else 1e-3)
    assert ms > 0.0
    d.close()


def test_sor_compare_leaves_the_next_step_unchanged():
    sc = city(nx=40, ny=24, nz=12, turb=0.1, fixed_sweeps=1, max_sweeps=10)
    rhs, p0 = _compatible_problem(sc, 4)
    a, b = les.Domain(sc), les.Domain(sc)
    a.step(1)
    b.step(1)
    a.sor_compare(les.LES_SOR_TWINNED, 0.9, 5, rhs, p0)
    a.sor_compare(les.LES_SOR_REDBLACK, -1.0, 5, rhs, p0)
    a.step(1)
    b.step(1)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    with pytest.raises(les.LesError):
        a.sor_compare(7, 0.9, 5, rhs, p0)
    a.close()
    b.close()
