"""Seeded synthetic inputs for the urban-flow LES time step.

This module builds the *inputs* of a time step and nothing else: the vertical
grid spacing, the building (solid-cell) mask, the log-law inflow profile that
stands in for the WRF wind profile of the paper's coupled runs (Sec. 4,
"Time synchronization and data exchange"), the initial velocity and the step
parameters.  It holds none of the method's arithmetic (no advection, no
viscosity, no Poisson operator), so both the FP64 CPU oracle and the CUDA
library consume exactly the same bytes from here.

Workloads (the paper's default domain is 150 x 150 x 90 with 50 SOR
iterations, Sec. 2.7 "Evaluation"; its WRF input files are not available, so
every input here is synthetic and seeded):

* ``lattice``   64x64x32, 16 cuboids on a 4x4 lattice (pitch 16, footprint
                 8x8 at offset 4, heights U(10,40) m), laminar log-law inflow,
                 exactly 50 SOR sweeps per step.
* ``random``    150x150x90, 100 random cuboids (sides U{4..16} rescaled to 30%
                 plan density, heights 20 m * exp(0.5 N(0,1))), 10% inflow
                 turbulence, SOR to relative residual 1e-6.
* ``large``     512x512x128, 1200 random cuboids, periodic in y.
* ``ensemble``  uneven domains 96^2..256^2 x 64..128, each with its own
                 buildings and log-law parameters.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

# boundary-condition codes (same numbering as the C header)
BC_INOUT = 0      # x: log-law inflow at x=0, zero-gradient outflow at x=L
BC_FREESLIP = 1   # y: free-slip side walls
BC_WALL = 2       # z: no-slip ground, free-slip lid
BC_PERIODIC = 3

KAPPA = 0.4       # von Karman constant used for the synthetic log-law inflow


@dataclasses.dataclass
class Scene:
    """One LES domain: grid, obstacles, inflow, initial state and step parameters."""

    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: np.ndarray            # (nz,) float64, cell heights in metres
    solid: np.ndarray         # (nz, ny, nx) uint8, 1 = building cell
    inflow_u: np.ndarray      # (nz,) float64, inflow profile at cell-centre heights
    bc_x: int = BC_INOUT
    bc_y: int = BC_FREESLIP
    bc_z: int = BC_WALL
    dt: float = 0.05
    cs: float = 0.1
    nu: float = 1.5e-5
    omega: float = 1.7
    tol: float = 1e-6
    max_sweeps: int = 50
    check_every: int = 10
    fixed_sweeps: int = 1
    turb: float = 0.0         # inflow turbulence intensity (fraction of U(z))
    seed: int = 0
    name: str = ""
    # initial state in I/O layout: u (nz, ny, nx+1), v (nz, ny+1, nx),
    # w (nz+1, ny, nx), p (nz, ny, nx)
    u0: Optional[np.ndarray] = None
    v0: Optional[np.ndarray] = None
    w0: Optional[np.ndarray] = None
    p0: Optional[np.ndarray] = None

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def params(self) -> dict:
        return dict(nx=self.nx, ny=self.ny, nz=self.nz, bc_x=self.bc_x, bc_y=self.bc_y,
                    bc_z=self.bc_z, dx=self.dx, dy=self.dy, dt=self.dt, cs=self.cs,
                    nu=self.nu, omega=self.omega, tol=self.tol, max_sweeps=self.max_sweeps,
                    check_every=self.check_every, fixed_sweeps=self.fixed_sweeps,
                    turb=self.turb, seed=self.seed)


# ----------------------------------------------------------------------------
# grid and inflow
# ----------------------------------------------------------------------------

def stretched_dz(nz: int, dz_min: float = 2.0, dz_max: float = 8.0) -> np.ndarray:
    """Geometric vertical spacing dz_k = dz_min * r^(k-1), r = (dz_max/dz_min)^(1/(nz-1))."""
    if nz == 1:
        return np.array([dz_min], dtype=np.float64)
    r = (dz_max / dz_min) ** (1.0 / (nz - 1))
    return dz_min * r ** np.arange(nz, dtype=np.float64)


def centre_heights(dz: np.ndarray) -> np.ndarray:
    """Height of each cell centre above the ground."""
    zw = np.cumsum(dz)
    return zw - 0.5 * dz


def log_law(z: np.ndarray, ustar: float, z0: float, kappa: float = KAPPA) -> np.ndarray:
    """Neutral log-law wind U(z) = (u*/kappa) ln(z/z0) for z > z0, else 0."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    m = z > z0
    out[m] = ustar / kappa * np.log(z[m] / z0)
    return out


# ----------------------------------------------------------------------------
# buildings
# ----------------------------------------------------------------------------

def rasterize(nx, ny, nz, dz, buildings, periodic_y=False) -> np.ndarray:
    """Solid mask: a cell is solid iff its centre lies inside a cuboid.

    ``buildings`` is a list of (x0, y0, sx, sy, H) in cell units / metres; the
    footprint covers cells [x0, x0+sx) x [y0, y0+sy) (y wraps when periodic).
    """
    zc = centre_heights(dz)
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    for (x0, y0, sx, sy, h) in buildings:
        ks = np.nonzero(zc < h)[0]
        if ks.size == 0:
            continue
        ys = np.arange(y0, y0 + sy)
        if periodic_y:
            ys = ys % ny
        for k in ks:
            solid[k][np.ix_(ys, np.arange(x0, x0 + sx))] = 1
    return solid


def lattice_buildings(rng, n_side=4, pitch=16, foot=8, offset=4, hmin=10.0, hmax=40.0):
    bs = []
    for b in range(n_side):
        for a in range(n_side):
            h = float(rng.uniform(hmin, hmax))
            bs.append((offset + pitch * a, offset + pitch * b, foot, foot, h))
    return bs


def random_buildings(rng, nx, ny, n_b, density=0.30, x_margin=16, gap=1,
                     periodic_y=False, side_lo=4, side_hi=16, h_median=20.0,
                     h_sigma=0.5, h_cap=None):
    """Random non-overlapping cuboids with a target plan density.

    Sides are drawn U{side_lo..side_hi}, then rescaled by a common factor until
    the total footprint is density*nx*ny within 1%; heights are lognormal with
    the given median and sigma.  Placement is by rejection with ``gap`` free
    cells between buildings and no building within ``x_margin`` cells of the
    inflow and outflow planes.
    """
    sides0 = rng.integers(side_lo, side_hi + 1, size=(n_b, 2)).astype(np.float64)
    heights = h_median * np.exp(h_sigma * rng.standard_normal(n_b))
    if h_cap is not None:
        heights = np.minimum(heights, h_cap)
    target = density * nx * ny

    def sides_for(scale):
        return np.maximum(1, np.rint(sides0 * scale)).astype(np.int64)

    # bisection on the common scale factor so the area is within 1% of target
    lo, hi = 0.05, 4.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        area = float(np.prod(sides_for(mid), axis=1).sum())
        if area < target:
            lo = mid
        else:
            hi = mid
    scale = hi

    for _attempt in range(50):
        sides = sides_for(scale)
        occ = np.zeros((ny, nx), dtype=bool)
        placed = []
        ok = True
        for b in range(n_b):
            sx, sy = int(sides[b, 0]), int(sides[b, 1])
            xlo, xhi = x_margin, nx - x_margin - sx
            if periodic_y:
                ylo, yhi = 0, ny - 1
            else:
                ylo, yhi = gap, ny - gap - sy
            if xhi < xlo or yhi < ylo:
                ok = False
                break
            done = False
            for _try in range(4000):
                x0 = int(rng.integers(xlo, xhi + 1))
                y0 = int(rng.integers(ylo, yhi + 1))
                ys = np.arange(y0 - gap, y0 + sy + gap)
                if periodic_y:
                    ys = ys % ny
                xs = np.arange(x0 - gap, x0 + sx + gap)
                if occ[np.ix_(ys, xs)].any():
                    continue
                ys_in = np.arange(y0, y0 + sy)
                if periodic_y:
                    ys_in = ys_in % ny
                occ[np.ix_(ys_in, np.arange(x0, x0 + sx))] = True
                placed.append((x0, y0, sx, sy, float(heights[b])))
                done = True
                break
            if not done:
                ok = False
                break
        if ok:
            return placed
        scale *= 0.98
    raise RuntimeError("could not place buildings")


# ----------------------------------------------------------------------------
# initial state
# ----------------------------------------------------------------------------

def initial_state(nx, ny, nz, solid, inflow_u):
    """u = inflow profile everywhere (zero on faces touching a building), v = w = p = 0."""
    u = np.broadcast_to(inflow_u[:, None, None], (nz, ny, nx + 1)).astype(np.float64).copy()
    # face i sits between cells i-1 and i (0-based cells); zero it if either is solid
    s = solid.astype(bool)
    touch = np.zeros((nz, ny, nx + 1), dtype=bool)
    touch[:, :, :nx] |= s
    touch[:, :, 1:] |= s
    u[touch] = 0.0
    v = np.zeros((nz, ny + 1, nx))
    w = np.zeros((nz + 1, ny, nx))
    p = np.zeros((nz, ny, nx))
    return u, v, w, p


def _finish(sc: Scene) -> Scene:
    sc.u0, sc.v0, sc.w0, sc.p0 = initial_state(sc.nx, sc.ny, sc.nz, sc.solid, sc.inflow_u)
    return sc


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def lattice_scene(seed: int = 0, nx=64, ny=64, nz=32, ustar=0.3, z0=0.1) -> Scene:
    """64x64x32 laminar case: 16 lattice cuboids, exactly 50 SOR sweeps per step."""
    rng = np.random.default_rng(seed)
    dz = stretched_dz(nz)
    bs = lattice_buildings(rng, n_side=max(1, min(nx, ny) // 16))
    solid = rasterize(nx, ny, nz, dz, bs)
    inflow = log_law(centre_heights(dz), ustar, z0)
    return _finish(Scene(nx=nx, ny=ny, nz=nz, dx=4.0, dy=4.0, dz=dz, solid=solid,
                         inflow_u=inflow, max_sweeps=50, fixed_sweeps=1, turb=0.0,
                         seed=seed, name=f"lattice_{nx}x{ny}x{nz}"))


def random_scene(seed: int = 0, nx=150, ny=150, nz=90, n_buildings=100, density=0.30,
                 ustar=0.3, z0=0.1, turb=0.1, periodic_y=False, tol=1e-6,
                 max_sweeps=20000, check_every=10, x_margin=16) -> Scene:
    """Random-city case (default 150x150x90, 100 cuboids, 10% inflow turbulence)."""
    rng = np.random.default_rng(seed)
    dz = stretched_dz(nz)
    ztop = float(np.sum(dz))
    bs = random_buildings(rng, nx, ny, n_buildings, density=density, x_margin=x_margin,
                          periodic_y=periodic_y, h_cap=0.6 * ztop)
    solid = rasterize(nx, ny, nz, dz, bs, periodic_y=periodic_y)
    inflow = log_law(centre_heights(dz), ustar, z0)
    return _finish(Scene(nx=nx, ny=ny, nz=nz, dx=4.0, dy=4.0, dz=dz, solid=solid,
                         inflow_u=inflow, bc_y=BC_PERIODIC if periodic_y else BC_FREESLIP,
                         tol=tol, max_sweeps=max_sweeps, check_every=check_every,
                         fixed_sweeps=0, turb=turb, seed=seed,
                         name=f"random_{nx}x{ny}x{nz}"))


def large_scene(seed: int = 0) -> Scene:
    """512x512x128, 1200 cuboids, periodic in y."""
    return random_scene(seed=seed, nx=512, ny=512, nz=128, n_buildings=1200,
                        periodic_y=True)


def ensemble_scenes(seed: int = 0, n: int = 32, turb: float = 0.1) -> List[Scene]:
    """Uneven domains: horizontal U{96..256}^2, vertical U{64..128}, own inflow each."""
    rng = np.random.default_rng(seed)
    out = []
    for d in range(n):
        nx = int(rng.integers(96, 257))
        ny = int(rng.integers(96, 257))
        nz = int(rng.integers(64, 129))
        ustar = float(rng.uniform(0.2, 0.6))
        z0 = float(rng.uniform(0.05, 0.5))
        nb = max(4, int(round(100 * nx * ny / (150 * 150))))
        sub_seed = int(rng.integers(0, 2**31 - 1))
        sc = random_scene(seed=sub_seed, nx=nx, ny=ny, nz=nz, n_buildings=nb, ustar=ustar,
                          z0=z0, turb=turb)
        sc.name = f"ens{d}_{nx}x{ny}x{nz}"
        out.append(sc)
    return out


def box_scene(nx, ny, nz, *, dx=4.0, dy=4.0, dz=None, bc=(BC_INOUT, BC_FREESLIP, BC_WALL),
              solid=None, inflow=None, **params) -> Scene:
    """A small custom domain for tests (no buildings unless ``solid`` is given)."""
    if dz is None:
        dz = np.full(nz, 4.0)
    dz = np.asarray(dz, dtype=np.float64)
    if solid is None:
        solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    if inflow is None:
        inflow = log_law(centre_heights(dz), 0.3, 0.1)
    sc = Scene(nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, solid=solid.astype(np.uint8),
               inflow_u=np.asarray(inflow, dtype=np.float64), bc_x=bc[0], bc_y=bc[1],
               bc_z=bc[2], **params)
    return _finish(sc)


def random_fields(sc: Scene, seed: int, amp: float = 1.0) -> Tuple[np.ndarray, ...]:
    """Seeded random velocity/pressure fields in I/O layout (for operator tests)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = sc.nx, sc.ny, sc.nz
    u = amp * rng.standard_normal((nz, ny, nx + 1))
    v = amp * rng.standard_normal((nz, ny + 1, nx))
    w = amp * rng.standard_normal((nz + 1, ny, nx))
    p = amp * rng.standard_normal((nz, ny, nx))
    return u, v, w, p


def random_rhs(sc: Scene, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal((sc.nz, sc.ny, sc.nx))
