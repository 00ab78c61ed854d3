"""Pins of the oracle's momentum routines (velfg, les, adam, feedbf, bondv1).

The paper prints only the u-component of velfg (Sec. 2.5); everything else is
a stated reading.  These tests pin each discrete term to a closed form it must
reproduce exactly (polynomial fields), and the whole step to invariants and to
the Taylor-Green exact solution of the Navier-Stokes equations."""

import numpy as np
import pytest

from oracle.oracle import (Oracle, A_U, A_V, A_W, A_P, A_NUT, A_FU, A_FV, A_FW)
from paper_1504_02264_gb300 import scene


# ----------------------------------------------------------------------------
# staggered coordinates of the padded arrays (index 0 and n+1 are ghosts)

def coords(sc):
    nx, ny, nz = sc.nx, sc.ny, sc.nz
    dzp = np.concatenate([[sc.dz[0]], sc.dz, [sc.dz[-1]]])       # mirrored ghost spacing
    zw = np.concatenate([[-dzp[0]], np.cumsum(np.concatenate([[0.0], dzp[1:]]))])
    # zw[m] is the top face of padded cell m-1 ... build explicitly:
    zw_face = np.zeros(nz + 2)          # top face of padded cell k (k = 0..nz+1)
    zw_face[0] = 0.0
    for k in range(1, nz + 2):
        zw_face[k] = zw_face[k - 1] + dzp[k]
    zc = zw_face - 0.5 * dzp            # centre of padded cell k
    xf = np.arange(nx + 2) * sc.dx      # east face of cell i
    xc = (np.arange(nx + 2) - 0.5) * sc.dx
    yf = np.arange(ny + 2) * sc.dy
    yc = (np.arange(ny + 2) - 0.5) * sc.dy
    return dict(xf=xf, xc=xc, yf=yf, yc=yc, zw=zw_face, zc=zc)


def grid3(x, y, z):
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def set_field(o, which, f, sc, stag):
    c = coords(sc)
    x = c["xf"] if stag == "u" else c["xc"]
    y = c["yf"] if stag == "v" else c["yc"]
    z = c["zw"] if stag == "w" else c["zc"]
    X, Y, Z = grid3(x, y, z)
    o.raw(which)[...] = f(X, Y, Z)
    return X, Y, Z


def zero(X, Y, Z):
    return np.zeros_like(X)


def interior_u(sc, a):
    return a[1:sc.nz + 1, 1:sc.ny + 1, 1:sc.nx]        # advanced u faces 1..nx-1


def interior_v(sc, a):
    return a[1:sc.nz + 1, 1:sc.ny, 1:sc.nx + 1]


def interior_w(sc, a):
    return a[1:sc.nz, 1:sc.ny + 1, 1:sc.nx + 1]


def run_tendency(sc, fu, fv, fw, sgs=False, nut=None):
    o = Oracle(sc)
    Xu = set_field(o, A_U, fu, sc, "u")
    Xv = set_field(o, A_V, fv, sc, "v")
    Xw = set_field(o, A_W, fw, sc, "w")
    if nut is not None:
        o.raw(A_NUT)[...] = nut
    o.tendency(with_sgs=sgs)
    return o, Xu, Xv, Xw


NU = 0.3


def mk(nx=8, ny=7, nz=6, stretched=False, **kw):
    dz = scene.stretched_dz(nz) if stretched else np.full(nz, 4.0)
    return scene.box_scene(nx, ny, nz, dz=dz, nu=NU, **kw)


# ----------------------------------------------------------------------------
# velfg: each advection / diffusion term against its closed form

def test_velfg_u_linear_x():
    """u = a x: advection u du/dx = a^2 x exactly (the printed cov1/covx form)."""
    sc = mk()
    a = 0.37
    o, (X, Y, Z), _, _ = run_tendency(sc, lambda X, Y, Z: a * X, zero, zero)
    np.testing.assert_allclose(interior_u(sc, o.raw(A_FU)), interior_u(sc, -a * a * X), rtol=1e-12, atol=1e-13)


def test_velfg_u_shear_y():
    """u = b y^2 advected by v = V: -2bVy + nu 2b (covy, diu2 terms)."""
    sc = mk()
    b, V = 0.013, 0.8
    o, (X, Y, Z), _, _ = run_tendency(sc, lambda X, Y, Z: b * Y * Y, lambda X, Y, Z: V + 0 * X, zero)
    exp = -2 * b * V * Y + NU * 2 * b
    np.testing.assert_allclose(interior_u(sc, o.raw(A_FU)), interior_u(sc, exp), rtol=1e-12, atol=1e-13)


def test_velfg_u_stretched_z():
    """u = c z advected by w = W on stretched dz: -Wc (cov3 with dzs)."""
    sc = mk(stretched=True)
    c, W = 0.05, -0.6
    o, (X, Y, Z), _, _ = run_tendency(sc, lambda X, Y, Z: c * Z, zero, lambda X, Y, Z: W + 0 * X)
    np.testing.assert_allclose(interior_u(sc, o.raw(A_FU)), -W * c, rtol=1e-12, atol=1e-13)


def test_velfg_u_diffusion_z_uniform():
    """u = b z^2 (uniform dz, w = 0): nu 2b (diu3 term)."""
    sc = mk()
    b = 0.02
    o, _, _, _ = run_tendency(sc, lambda X, Y, Z: b * Z * Z, zero, zero)
    np.testing.assert_allclose(interior_u(sc, o.raw(A_FU)), NU * 2 * b, rtol=1e-12)


def test_velfg_v_terms():
    sc = mk()
    a = 0.21
    o, _, (X, Y, Z), _ = run_tendency(sc, zero, lambda X, Y, Z: a * Y, zero)
    np.testing.assert_allclose(interior_v(sc, o.raw(A_FV)), interior_v(sc, -a * a * Y), rtol=1e-12, atol=1e-13)
    b, U = 0.011, 1.3
    o, _, (X, Y, Z), _ = run_tendency(sc, lambda X, Y, Z: U + 0 * X, lambda X, Y, Z: b * X * X, zero)
    exp = -2 * b * U * X + NU * 2 * b
    np.testing.assert_allclose(interior_v(sc, o.raw(A_FV)), interior_v(sc, exp), rtol=1e-12, atol=1e-13)
    scs = mk(stretched=True)
    c, W = 0.07, 0.4
    o, _, _, _ = run_tendency(scs, zero, lambda X, Y, Z: c * Z, lambda X, Y, Z: W + 0 * X)
    np.testing.assert_allclose(interior_v(scs, o.raw(A_FV)), -W * c, rtol=1e-12)


def test_velfg_w_terms():
    scs = mk(stretched=True)
    a = 0.09
    o, _, _, (X, Y, Z) = run_tendency(scs, zero, zero, lambda X, Y, Z: a * Z)
    # own-direction advection: dz-weighted interpolation of cov to the face
    np.testing.assert_allclose(interior_w(scs, o.raw(A_FW)), interior_w(scs, -a * a * Z), rtol=1e-12, atol=1e-13)
    b, U = 0.017, 0.9
    o, _, _, (X, Y, Z) = run_tendency(scs, lambda X, Y, Z: U + 0 * X, zero, lambda X, Y, Z: b * X * X)
    exp = -2 * b * U * X + NU * 2 * b
    np.testing.assert_allclose(interior_w(scs, o.raw(A_FW)), interior_w(scs, exp), rtol=1e-12, atol=1e-13)
    V = -0.7
    o, _, _, (X, Y, Z) = run_tendency(scs, zero, lambda X, Y, Z: V + 0 * X, lambda X, Y, Z: b * Y * Y)
    exp = -2 * b * V * Y + NU * 2 * b
    np.testing.assert_allclose(interior_w(scs, o.raw(A_FW)), interior_w(scs, exp), rtol=1e-12, atol=1e-13)
    # advecting u interpolated in z with dz weights: u = c z gives ubar = c z_w
    c = 0.3
    o, _, _, (X, Y, Z) = run_tendency(scs, lambda X, Y, Z: c * Z, zero, lambda X, Y, Z: 0.05 * X)
    exp = -(c * Z) * 0.05
    np.testing.assert_allclose(interior_w(scs, o.raw(A_FW)), interior_w(scs, exp), rtol=1e-12, atol=1e-13)


# ----------------------------------------------------------------------------
# les: Smagorinsky viscosity and SGS stress divergence

def _nut_interior(o, sc):
    return o.raw(A_NUT)[1:sc.nz + 1, 1:sc.ny + 1, 1:sc.nx + 1]


@pytest.mark.parametrize("case", ["shear_y", "shear_z_stretched", "strain"])
def test_smagorinsky_closed_form(case):
    """|S| of simple flows: pure shear gives |S| = gamma; plane strain 2a."""
    cs = 0.1
    if case == "shear_y":
        sc = mk(cs=cs)
        g = 0.4
        fu, fv, fw, smag = (lambda X, Y, Z: g * Y), zero, zero, g
    elif case == "shear_z_stretched":
        sc = mk(stretched=True, cs=cs)
        g = 0.25
        fu, fv, fw, smag = (lambda X, Y, Z: g * Z), zero, zero, g
    else:
        sc = mk(cs=cs)
        a = 0.3
        fu, fv, fw, smag = (lambda X, Y, Z: a * X), (lambda X, Y, Z: -a * Y), zero, 2 * a
    o = Oracle(sc)
    set_field(o, A_U, fu, sc, "u")
    set_field(o, A_V, fv, sc, "v")
    set_field(o, A_W, fw, sc, "w")
    o.les_nut()
    delta = (sc.dx * sc.dy * sc.dz) ** (1.0 / 3.0)
    exp = ((cs * delta) ** 2 * smag)[:, None, None] * np.ones((sc.nz, sc.ny, sc.nx))
    np.testing.assert_allclose(_nut_interior(o, sc), exp, rtol=1e-12)


@pytest.mark.parametrize("comp", ["u_y", "u_z", "v_x", "w_y"])
def test_sgs_constant_viscosity(comp):
    """With a constant nu_t the SGS force of a parabolic profile is 2 b nu_t."""
    sc = mk()
    nut = 0.7
    b = 0.015
    f = {"u_y": (lambda X, Y, Z: b * Y * Y, zero, zero),
         "u_z": (lambda X, Y, Z: b * Z * Z, zero, zero),
         "v_x": (zero, lambda X, Y, Z: b * X * X, zero),
         "w_y": (zero, zero, lambda X, Y, Z: b * Y * Y)}[comp]
    o1, _, _, _ = run_tendency(sc, *f, sgs=True, nut=nut)
    o0, _, _, _ = run_tendency(sc, *f, sgs=False)
    which, sel = {"u": (A_FU, interior_u), "v": (A_FV, interior_v), "w": (A_FW, interior_w)}[comp[0]]
    d = sel(sc, o1.raw(which)) - sel(sc, o0.raw(which))
    np.testing.assert_allclose(d, 2 * b * nut, rtol=1e-11)


def test_sgs_dissipative_periodic():
    """Sum over faces of u . F_sgs is negative for a random periodic field."""
    n = 8
    sc = scene.box_scene(n, n, n, dz=np.full(n, 4.0),
                         bc=(scene.BC_PERIODIC, scene.BC_PERIODIC, scene.BC_PERIODIC), cs=0.2)
    rng = np.random.default_rng(1)
    u, v, w, p = scene.random_fields(sc, 4)
    u[:, :, 0] = u[:, :, -1]
    v[:, 0, :] = v[:, -1, :]
    w[0] = w[-1]
    o = Oracle(sc)
    o.set_fields(u, v, w, p)
    o.bc_fill()
    o.les_nut()
    o.tendency(with_sgs=True)
    f1 = [o.raw(a).copy() for a in (A_FU, A_FV, A_FW)]
    o.tendency(with_sgs=False)
    f0 = [o.raw(a).copy() for a in (A_FU, A_FV, A_FW)]
    sl = (slice(1, n + 1),) * 3
    diss = sum(np.sum(o.raw(a)[sl] * (g1[sl] - g0[sl])) for a, g1, g0 in zip((A_U, A_V, A_W), f1, f0))
    assert diss < 0.0
    assert np.all(o.raw(A_NUT)[sl] > 0)


# ----------------------------------------------------------------------------
# whole-step invariants

def _tg_scene(n, nu, dt, cs=0.0):
    L = 2 * np.pi
    h = L / n
    sc = scene.box_scene(n, n, 2, dx=h, dy=h, dz=np.full(2, h),
                         bc=(scene.BC_PERIODIC, scene.BC_PERIODIC, scene.BC_PERIODIC),
                         nu=nu, dt=dt, cs=cs, fixed_sweeps=0, tol=1e-12, max_sweeps=20000,
                         check_every=10)
    c = coords(sc)
    Xu, Yu, _ = grid3(c["xf"][1:n + 1], c["yc"][1:n + 1], c["zc"][1:3])
    Xv, Yv, _ = grid3(c["xc"][1:n + 1], c["yf"][1:n + 1], c["zc"][1:3])
    u = np.sin(Xu) * np.cos(Yu)
    v = -np.cos(Xv) * np.sin(Yv)
    uu = np.concatenate([u[:, :, -1:], u], axis=2)          # face 0 == face n
    vv = np.concatenate([v[:, -1:, :], v], axis=1)
    ww = np.zeros((3, n, n))
    return sc, uu, vv, ww


def _ke(o):
    u, v, w, _ = o.fields()
    return 0.5 * (np.sum(u[:, :, 1:] ** 2) + np.sum(v[:, 1:, :] ** 2) + np.sum(w[1:] ** 2))


def _tg_run(n, nu, dt, T, cs=0.0, record=False):
    sc, u, v, w = _tg_scene(n, nu, dt, cs)
    o = Oracle(sc)
    o.set_fields(u, v, w, np.zeros((2, n, n)))
    ke0 = _ke(o)
    hist = [1.0]
    for _ in range(int(round(T / dt))):
        o.step(1)
        if record:
            hist.append(_ke(o) / ke0)
    return (_ke(o) / ke0, hist) if record else _ke(o) / ke0


def test_taylor_green_decay():
    """2-D Taylor-Green vortex (exact NS solution): KE decays as exp(-4 nu t),
    with the decay rate of the discrete Laplacian on the grid."""
    n, nu, dt, T = 16, 0.05, 0.02, 1.0
    h = 2 * np.pi / n
    lam = 2 * (2 - 2 * np.cos(h)) / h ** 2       # -> 2 (= |k|^2) as h -> 0
    r = _tg_run(n, nu, dt, T)
    exp = np.exp(-2 * nu * lam * T)
    assert abs(r - exp) < 2e-3 * exp, (r, exp)
    assert abs(r - np.exp(-4 * nu * T)) < 2e-2


def test_taylor_green_second_order_in_time():
    """Adams-Bashforth 2: the time error falls ~4x when dt halves."""
    n, nu, T = 16, 0.1, 0.8
    rs = [_tg_run(n, nu, dt, T) for dt in (0.04, 0.02, 0.01)]
    q = (rs[0] - rs[1]) / (rs[1] - rs[2])
    assert 3.0 < q < 5.0, (rs, q)


def test_taylor_green_smagorinsky_monotone():
    n, nu, dt, T = 16, 0.01, 0.02, 0.6
    r0 = _tg_run(n, nu, dt, T, cs=0.0)
    r1, hist = _tg_run(n, nu, dt, T, cs=0.17, record=True)
    assert np.all(np.diff(hist) < 0)
    assert r1 < r0


def test_uniform_flow_periodic_stays_uniform():
    n = 6
    sc = scene.box_scene(n, n, n, dz=np.full(n, 4.0),
                         bc=(scene.BC_PERIODIC, scene.BC_PERIODIC, scene.BC_PERIODIC),
                         fixed_sweeps=1, max_sweeps=5)
    o = Oracle(sc)
    u = np.full((n, n, n + 1), 1.0)
    v = np.full((n, n + 1, n), 0.5)
    w = np.full((n + 1, n, n), 0.2)
    o.set_fields(u, v, w, np.zeros((n, n, n)))
    o.step(3)
    uu, vv, ww, pp = o.fields()
    assert np.all(o.get(A_NUT) == 0.0)
    np.testing.assert_allclose(uu, 1.0, atol=1e-14)
    np.testing.assert_allclose(vv, 0.5, atol=1e-14)
    np.testing.assert_allclose(ww, 0.2, atol=1e-14)


def test_rest_stays_at_rest():
    sc = scene.lattice_scene(0, nx=32, ny=32, nz=16)
    sc.inflow_u = np.zeros_like(sc.inflow_u)
    o = Oracle(sc)
    z = [np.zeros_like(a) for a in (sc.u0, sc.v0, sc.w0, sc.p0)]
    o.set_fields(*z)
    o.step(2)
    for a in o.fields():
        assert np.all(a == 0.0)


def test_mirror_symmetry_y():
    """A y-mirror-symmetric layout (odd ny, so the mirror keeps the SOR colours)
    keeps u, w, p symmetric and v antisymmetric."""
    nx, ny, nz = 24, 15, 10
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:4, 4:11, 8:12] = 1           # centred in y
    solid[:6, 1:3, 16:18] = 1
    solid[:6, ny - 3:ny - 1, 16:18] = 1
    sc = scene.box_scene(nx, ny, nz, dz=scene.stretched_dz(nz), solid=solid,
                         fixed_sweeps=1, max_sweeps=30)
    o = Oracle(sc)
    o.step(3)
    u, v, w, p = o.fields()
    s = max(np.abs(u).max(), 1.0)
    np.testing.assert_allclose(u, u[:, ::-1, :], atol=1e-12 * s)
    np.testing.assert_allclose(w, w[:, ::-1, :], atol=1e-12 * s)
    np.testing.assert_allclose(v, -v[:, ::-1, :], atol=1e-12 * s)
    np.testing.assert_allclose(p, p[:, ::-1, :], atol=1e-12 * max(np.abs(p).max(), 1.0))


def test_mass_flux_balanced_after_correction():
    sc = scene.lattice_scene(1, nx=32, ny=32, nz=16)
    o = Oracle(sc)
    o.step(2)
    st = o.stats()
    assert abs(st["q_out"] - st["q_in"]) <= 1e-12 * abs(st["q_in"])
    assert st["mass_factor"] != 1.0


# ----------------------------------------------------------------------------
# axis exchange: on a uniform, all-periodic cube the readings of v and w (not
# printed in the paper) must be the printed u-formula with the axes exchanged

def _periodic_raw(n, rng):
    """A random field on the padded (n+2)^3 array whose ghosts hold the
    periodic images (index 0 = n, n+1 = 1 on every axis)."""
    a = rng.standard_normal((n, n, n))
    idx = (np.arange(n + 2) - 1) % n
    return a[np.ix_(idx, idx, idx)]


@pytest.mark.parametrize("sgs", [False, True])
@pytest.mark.parametrize("swap", ["xy", "xz"])
def test_tendency_axis_exchange(swap, sgs):
    """Exchanging two axes of the flow (velocity components and coordinates)
    exchanges the corresponding tendencies: pins the v and w advection,
    diffusion and SGS readings against the printed u formula."""
    n = 6
    per = (scene.BC_PERIODIC,) * 3
    # unequal spacings, exchanged with the axes (a dx / dy / dz mix-up in a
    # reading breaks the symmetry); dz uniform so that z can trade with x
    sp = {"xy": ((3.0, 5.0, 4.0), (5.0, 3.0, 4.0)), "xz": ((3.0, 4.0, 5.0), (5.0, 4.0, 3.0))}[swap]
    scenes = [scene.box_scene(n, n, n, dx=a, dy=b, dz=np.full(n, c), bc=per, nu=NU) for a, b, c in sp]
    rng = np.random.default_rng(12)
    u, v, w, nut = (_periodic_raw(n, rng) for _ in range(4))
    nut = np.abs(nut)
    if swap == "xy":
        t = lambda a: np.transpose(a, (0, 2, 1))        # [k, j, i] -> [k, i, j]
        u2, v2, w2 = t(v), t(u), t(w)
    else:
        t = lambda a: np.transpose(a, (2, 1, 0))        # [k, j, i] -> [i, j, k]
        u2, v2, w2 = t(w), t(v), t(u)

    def tend(sc, uu, vv, ww, nn):
        o = Oracle(sc)
        o.raw(A_U)[...] = uu
        o.raw(A_V)[...] = vv
        o.raw(A_W)[...] = ww
        o.raw(A_NUT)[...] = nn
        o.tendency(with_sgs=sgs)
        s = slice(1, n + 1)
        return [o.raw(a)[s, s, s].copy() for a in (A_FU, A_FV, A_FW)]

    fu, fv, fw = tend(scenes[0], u, v, w, nut)
    gu, gv, gw = tend(scenes[1], u2, v2, w2, t(nut))
    scale = max(np.abs(f).max() for f in (fu, fv, fw))
    if swap == "xy":
        pairs = ((gu, t(fv)), (gv, t(fu)), (gw, t(fw)))
    else:
        pairs = ((gu, t(fw)), (gv, t(fv)), (gw, t(fu)))
    for got, want in pairs:
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * scale)


# ----------------------------------------------------------------------------
# wall ghosts (bondv1 reading): no-slip at the ground face, free slip at the
# lid and at the side walls, each against the closed form it makes exact

def _wall_scene():
    # x periodic so that the inflow plays no part; y free-slip walls; z ground + lid
    return scene.box_scene(6, 5, 7, dz=np.full(7, 3.0), nu=NU,
                           bc=(scene.BC_PERIODIC, scene.BC_FREESLIP, scene.BC_WALL))


def _filled_tendency(sc, fu, fv, fw):
    o = Oracle(sc)
    set_field(o, A_U, fu, sc, "u")
    set_field(o, A_V, fv, sc, "v")
    set_field(o, A_W, fw, sc, "w")
    o.bc_fill()
    o.tendency(with_sgs=False)
    return o


def test_ground_no_slip_at_the_face():
    """u = a z vanishes on the ground face: with the ground ghost = -u(1) the
    linear profile continues through the face and its discrete diffusion is 0
    in the first cell too (a no-slip point at the first centre would not give
    this)."""
    sc = _wall_scene()
    a = 0.13
    o = _filled_tendency(sc, lambda X, Y, Z: a * Z, zero, zero)
    fu = o.raw(A_FU)[1:sc.nz, 1:sc.ny + 1, 1:sc.nx + 1]        # the lid cell feels the free-slip lid
    np.testing.assert_allclose(fu, 0.0, atol=1e-14)


def test_lid_free_slip_mirror():
    """u = b (z - H)^2 is symmetric about the lid face z = H: the free-slip
    mirror ghost makes the discrete diffusion exact (2 nu b) up to the lid cell."""
    sc = _wall_scene()
    H = float(np.sum(sc.dz))
    b = 0.021
    o = _filled_tendency(sc, lambda X, Y, Z: b * (Z - H) ** 2, zero, zero)
    fu = o.raw(A_FU)[2:sc.nz + 1, 1:sc.ny + 1, 1:sc.nx + 1]     # cell 1 feels the no-slip ground
    np.testing.assert_allclose(fu, 2 * NU * b, rtol=1e-12)


def test_side_wall_free_slip_mirror():
    """u = b y^2 is symmetric about the side wall y = 0: the free-slip mirror
    ghost makes the discrete y-diffusion exact (2 nu b) in the first row."""
    sc = _wall_scene()
    b = 0.017
    o = _filled_tendency(sc, lambda X, Y, Z: b * Y * Y, zero, zero)
    fu = o.raw(A_FU)[2:sc.nz + 1, 1:3, 1:sc.nx + 1]             # cell k = 1 feels the no-slip ground
    np.testing.assert_allclose(fu, 2 * NU * b, rtol=1e-12)
