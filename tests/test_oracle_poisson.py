"""Pins of the oracle's pressure solver (routine press, Sec. 2.6) against
textbook matrices, direct solves, manufactured solutions and the matrix form of
SOR.  None of these re-types the oracle's stencil: every expected value comes
from a different construction (Kronecker sums, a graph Laplacian, LAPACK, a
continuous solution, the textbook SOR recurrence on an assembled matrix)."""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph

from oracle.oracle import Oracle, A_P, A_RHS
from paper_1504_02264_gb300 import scene


def assemble(o: Oracle, nx, ny, nz):
    """Dense matrix of the oracle's operator, column by column (A e_m)."""
    n = nx * ny * nz
    A = np.zeros((n, n))
    e = np.zeros(n)
    for m in range(n):
        e[:] = 0.0
        e[m] = 1.0
        A[:, m] = o.apply_A(e.reshape(nz, ny, nx)).ravel()
    return A


def lap1d(n, h, periodic=False):
    L = np.zeros((n, n))
    for a in range(n):
        if a > 0:
            L[a, a - 1] = 1
        if a < n - 1:
            L[a, a + 1] = 1
    if periodic:
        L[0, n - 1] = L[n - 1, 0] = 1
    L -= np.diag(L.sum(axis=1))
    return L / h ** 2


@pytest.mark.parametrize("periodic_y", [False, True])
def test_textbook_laplacian_uniform(periodic_y):
    nx, ny, nz = 5, 4, 3
    dx, dy, dz = 2.0, 3.0, 1.5
    sc = scene.box_scene(nx, ny, nz, dx=dx, dy=dy, dz=np.full(nz, dz),
                         bc=(scene.BC_INOUT, scene.BC_PERIODIC if periodic_y else scene.BC_FREESLIP,
                             scene.BC_WALL))
    o = Oracle(sc)
    A = assemble(o, nx, ny, nz)
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    Aexp = (np.kron(np.kron(lap1d(nz, dz), Iy), Ix) +
            np.kron(np.kron(Iz, lap1d(ny, dy, periodic_y)), Ix) +
            np.kron(np.kron(Iz, Iy), lap1d(nx, dx)))
    np.testing.assert_allclose(A, Aexp, rtol=0, atol=1e-14)


def test_graph_laplacian_with_buildings():
    """Uniform spacing h: A on fluid cells is minus the graph Laplacian / h^2."""
    nx, ny, nz, h = 7, 6, 5, 2.0
    rng = np.random.default_rng(3)
    solid = (rng.random((nz, ny, nx)) < 0.25).astype(np.uint8)
    sc = scene.box_scene(nx, ny, nz, dx=h, dy=h, dz=np.full(nz, h), solid=solid)
    o = Oracle(sc)
    A = assemble(o, nx, ny, nz)
    fluid = solid.ravel() == 0
    n = nx * ny * nz
    rows, cols = [], []
    idx = np.arange(n).reshape(nz, ny, nx)
    for axis in range(3):
        a = np.take(idx, range(0, idx.shape[axis] - 1), axis=axis).ravel()
        b = np.take(idx, range(1, idx.shape[axis]), axis=axis).ravel()
        keep = fluid[a] & fluid[b]
        rows += [a[keep], b[keep]]
        cols += [b[keep], a[keep]]
    adj = sp.coo_matrix((np.ones(sum(len(r) for r in rows)), (np.concatenate(rows), np.concatenate(cols))),
                        shape=(n, n)).toarray()
    L = csgraph.laplacian(adj)
    # isolated fluid cells (no open face) are not unknowns
    active = fluid & (adj.sum(axis=1) > 0)
    Aexp = np.where(active[:, None], -L / h ** 2, 0.0)
    np.testing.assert_allclose(A, Aexp, rtol=0, atol=1e-14)


def test_stretched_volume_symmetry_and_null_space():
    """On stretched dz, V A is symmetric (V = dz_k) and A 1 = 0."""
    nx, ny, nz = 6, 5, 6
    rng = np.random.default_rng(5)
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:3, 1:3, 2:4] = 1
    sc = scene.box_scene(nx, ny, nz, dz=scene.stretched_dz(nz), solid=solid)
    o = Oracle(sc)
    A = assemble(o, nx, ny, nz)
    V = np.repeat(sc.dz, nx * ny)
    VA = V[:, None] * A
    np.testing.assert_allclose(VA, VA.T, rtol=0, atol=1e-14)
    np.testing.assert_allclose(A @ np.ones(A.shape[0]), 0.0, atol=1e-14)


def _vmean(p, dz, fluid):
    w = np.broadcast_to(dz[:, None, None], p.shape)[fluid]
    return np.sum(w * p[fluid]) / np.sum(w)


def test_dense_solve_6x6x6():
    """SOR converges to the LAPACK least-squares solution of the gauge-fixed system."""
    n = 6
    solid = np.zeros((n, n, n), np.uint8)
    solid[:2, 1:3, 1:3] = 1
    solid[:4, 4, 4] = 1
    dz = scene.stretched_dz(n)
    sc = scene.box_scene(n, n, n, dz=dz, solid=solid, fixed_sweeps=1, max_sweeps=4000)
    o = Oracle(sc)
    A = assemble(o, n, n, n)
    fluid = solid == 0
    rng = np.random.default_rng(11)
    rhs = rng.standard_normal((n, n, n)) * fluid
    rhs[fluid] -= _vmean(rhs, dz, fluid)
    f = fluid.ravel()
    Af = A[np.ix_(f, f)]
    x = np.linalg.lstsq(Af, rhs.ravel()[f], rcond=None)[0]
    pd = np.zeros(n ** 3)
    pd[f] = x
    pd = pd.reshape(n, n, n)
    pd[fluid] -= _vmean(pd, dz, fluid)
    o.set(A_P, np.zeros((n, n, n)))
    o.pressure_solve(rhs)
    p = o.get(A_P)
    assert o.stats()["rel_residual"] < 1e-13
    np.testing.assert_allclose(p, pd, rtol=0, atol=1e-12 * np.abs(pd).max())


def test_manufactured_discrete():
    """rhs = A p_exact recovers p_exact (up to the gauge)."""
    nx, ny, nz = 9, 7, 8
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:5, 2:4, 3:6] = 1
    dz = scene.stretched_dz(nz)
    sc = scene.box_scene(nx, ny, nz, dz=dz, solid=solid, fixed_sweeps=0, tol=1e-13,
                         max_sweeps=20000, check_every=10)
    o = Oracle(sc)
    fluid = solid == 0
    rng = np.random.default_rng(2)
    pex = rng.standard_normal((nz, ny, nx)) * fluid
    pex[fluid] -= _vmean(pex, dz, fluid)
    rhs = o.apply_A(pex)
    o.set(A_P, np.zeros_like(pex))
    o.pressure_solve(rhs)
    st = o.stats()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-13
    np.testing.assert_allclose(o.get(A_P), pex, rtol=0, atol=1e-10)


def test_manufactured_continuous_second_order_uniform():
    """p = cos(pi x/Lx) cos(pi y/Ly) cos(pi z/Lz): error falls ~4x per refinement."""
    errs = []
    for n in (8, 16, 32):
        nx = ny = n
        nz = n // 2
        dx = dy = 8.0 / n
        dz = np.full(nz, 8.0 / n)
        Lx, Ly, Lz = nx * dx, ny * dy, float(dz.sum())
        xc = (np.arange(nx) + 0.5) * dx
        yc = (np.arange(ny) + 0.5) * dy
        zc = np.cumsum(dz) - 0.5 * dz
        Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
        pex = np.cos(np.pi * X / Lx) * np.cos(np.pi * Y / Ly) * np.cos(np.pi * Z / Lz)
        rhs = -np.pi ** 2 * (1 / Lx ** 2 + 1 / Ly ** 2 + 1 / Lz ** 2) * pex
        omega = 2.0 / (1.0 + np.sin(np.pi / n))
        sc = scene.box_scene(nx, ny, nz, dx=dx, dy=dy, dz=dz, fixed_sweeps=0, tol=1e-11,
                             max_sweeps=50000, check_every=20, omega=omega)
        o = Oracle(sc)
        o.pressure_solve(rhs)
        assert o.stats()["status"] == 0
        p = o.get(A_P)
        pe = pex - _vmean(pex, dz, np.ones_like(p, dtype=bool))
        errs.append(np.abs(p - pe).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs


def test_manufactured_continuous_second_order_stretched():
    """Stretched z (nested refinement of z(xi) = Lz (e^{a xi}-1)/(e^a-1), a = ln 4,
    top cells ~4x the bottom ones like the LES grids), p = cos(pi z/Lz): the error
    ratio per refinement rises towards 4 (second order, supra-convergent)."""
    errs = []
    for nz in (16, 32, 64):
        nx = ny = 4
        a = np.log(4.0)
        zw = 4.0 * (np.exp(a * np.arange(nz + 1) / nz) - 1.0) / (np.exp(a) - 1.0)
        dz = np.diff(zw)
        Lz = float(dz.sum())
        zc = np.cumsum(dz) - 0.5 * dz
        pex = np.cos(np.pi * zc / Lz)[:, None, None] * np.ones((nz, ny, nx))
        rhs = -np.pi ** 2 / Lz ** 2 * pex
        sc = scene.box_scene(nx, ny, nz, dx=1.0, dy=1.0, dz=dz, fixed_sweeps=0, tol=1e-12,
                             max_sweeps=200000, check_every=50, omega=1.9)
        o = Oracle(sc)
        o.pressure_solve(rhs)
        assert o.stats()["status"] == 0
        p = o.get(A_P)
        pe = pex - _vmean(pex, dz, np.ones_like(p, dtype=bool))
        errs.append(np.abs(p - pe).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < r2 < 4.2, errs


def test_colour_order_first_half_sweep():
    """nrd = 0 updates exactly the cells with i+j+k odd (1-based)."""
    n = 3
    sc = scene.box_scene(n, n, n)
    o = Oracle(sc)
    rng = np.random.default_rng(0)
    p0 = rng.standard_normal((n, n, n))
    o.set(A_P, p0)
    o.set(A_RHS, rng.standard_normal((n, n, n)))
    o.sor_half(0)
    p1 = o.get(A_P)
    k, j, i = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    odd = (i + j + k) % 2 == 1
    assert np.all(p1[~odd] == p0[~odd])
    assert np.all(p1[odd] != p0[odd])


@pytest.mark.parametrize("omega", [1.0, 1.7])
def test_matrix_form_sor(omega):
    """Three red-black sweeps equal textbook SOR on the assembled matrix with the
    unknowns ordered odd-parity cells first, then even (lexicographic k, j, i)."""
    nx, ny, nz = 4, 5, 3
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[0, 2, 1] = 1
    sc = scene.box_scene(nx, ny, nz, dz=scene.stretched_dz(nz), solid=solid, omega=omega)
    o = Oracle(sc)
    A = assemble(o, nx, ny, nz)
    rng = np.random.default_rng(7)
    p0 = rng.standard_normal((nz, ny, nx)) * (solid == 0)
    b = rng.standard_normal((nz, ny, nx)) * (solid == 0)
    o.set(A_P, p0)
    o.set(A_RHS, b)
    o.sor_sweeps(3)
    got = o.get(A_P).ravel()
    k, j, i = np.meshgrid(np.arange(1, nz + 1), np.arange(1, ny + 1), np.arange(1, nx + 1), indexing="ij")
    par = ((i + j + k) % 2).ravel()
    order = [m for m in range(A.shape[0]) if par[m] == 1] + [m for m in range(A.shape[0]) if par[m] == 0]
    x = p0.ravel().copy()
    bb = b.ravel()
    for _ in range(3):
        for m in order:
            if A[m, m] == 0.0:
                continue
            s = A[m] @ x - A[m, m] * x[m]
            x[m] = x[m] + omega * ((bb[m] - s) / A[m, m] - x[m])
    np.testing.assert_allclose(got, x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("omega", [0.6, 0.9])
def test_twinned_sweep_is_two_jacobi_steps(omega):
    """One twinned double-buffer sweep (Sec. 2.6: the second copy from the
    first, then the first from the second) equals two steps of the textbook
    weighted Jacobi recurrence on the assembled matrix, every unknown updated
    from the previous iterate only."""
    nx, ny, nz = 4, 5, 3
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[0, 2, 1] = 1
    sc = scene.box_scene(nx, ny, nz, dz=scene.stretched_dz(nz), solid=solid)
    o = Oracle(sc)
    A = assemble(o, nx, ny, nz)
    rng = np.random.default_rng(9)
    p0 = rng.standard_normal((nz, ny, nx)) * (solid == 0)
    b = rng.standard_normal((nz, ny, nx)) * (solid == 0)
    o.set(A_P, p0)
    o.set(A_RHS, b)
    o.twin_sweeps(2, omega)
    got = o.get(A_P).ravel()
    x = p0.ravel().copy()
    bb = b.ravel()
    d = np.diag(A)
    live = d != 0.0
    for _ in range(4):
        s = A @ x - d * x
        xn = x.copy()
        xn[live] = x[live] + omega * ((bb[live] - s[live]) / d[live] - x[live])
        x = xn
    np.testing.assert_allclose(got, x, rtol=0, atol=1e-13)


def test_twinned_relaxation_range():
    """The twinned scheme is a weighted Jacobi iteration: on a compatible
    problem it converges for a relaxation below 1 and diverges at the SOR value
    1.7 (the iteration multiplies the checkerboard mode by about 1 - 2 omega)."""
    n = 8
    solid = np.zeros((n, n, n), np.uint8)
    solid[:3, 2:4, 2:4] = 1
    solid[:5, 5, 5] = 1
    dz = scene.stretched_dz(n)
    sc = scene.box_scene(n, n, n, dz=dz, solid=solid)
    fluid = solid == 0
    rng = np.random.default_rng(5)
    rhs = rng.standard_normal((n, n, n)) * fluid
    rhs[fluid] -= _vmean(rhs, dz, fluid)
    res = {}
    for omega, sweeps in ((0.9, 100), (1.7, 30)):
        o = Oracle(sc)
        o.set(A_P, np.zeros((n, n, n)))
        o.set(A_RHS, rhs)
        r0 = o.residual()
        o.twin_sweeps(sweeps, omega)
        res[omega] = o.residual() / r0
    assert res[0.9] < 1e-2
    assert res[1.7] > 1e6
