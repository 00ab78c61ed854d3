"""CPU-side checks of the C ABI: the library builds, loads, exports every
symbol that include/les.h declares, and rejects bad grids on the host (no GPU
work happens before validation)."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_1504_02264_gb300 import build as lesbuild
from paper_1504_02264_gb300 import les, scene

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(les_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libles():
    lesbuild.build()
    return les.lib()


def test_exports_every_declared_symbol(libles):
    names = declared_functions()
    assert {"les_create", "les_step", "les_pressure_solve", "les_get_fields"} <= names
    for n in sorted(names):
        assert hasattr(libles, n), n


def test_version(libles):
    assert "sm_103a" in les.les_version()


def _grid(sc, **kw):
    dz = np.ascontiguousarray(sc.dz)
    g = les.les_grid_t(nx=sc.nx, ny=sc.ny, nz=sc.nz, bc_x=sc.bc_x, bc_y=sc.bc_y, bc_z=sc.bc_z,
                       dx=sc.dx, dy=sc.dy, dz=dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       dt=sc.dt, cs=sc.cs, nu=sc.nu, omega=sc.omega, tol=sc.tol,
                       max_sweeps=sc.max_sweeps, check_every=sc.check_every,
                       fixed_sweeps=sc.fixed_sweeps, precision=0, turb=sc.turb, seed=sc.seed)
    for k, v in kw.items():
        setattr(g, k, v)
    return g, dz


@pytest.mark.parametrize("bad", [dict(nx=1), dict(omega=2.0), dict(omega=0.0), dict(bc_y=7),
                                 dict(bc_x=les.LES_BC_PERIODIC, nx=9), dict(max_sweeps=0),
                                 dict(precision=5), dict(dt=0.0), dict(bc_z=les.LES_BC_FREESLIP)])
def test_create_rejects_bad_grids_on_host(libles, bad):
    sc = scene.box_scene(10, 8, 6)
    g, dz = _grid(sc, **bad)
    solid = np.zeros((g.nz, g.ny, g.nx), np.uint8)
    h = ctypes.c_void_p()
    rc = libles.les_create(ctypes.byref(g), solid.ctypes.data, sc.inflow_u.ctypes.data, None, ctypes.byref(h))
    assert rc == les.LES_EINVAL
    assert h.value is None
    assert les.les_last_error(None)


def test_null_handle_is_einval(libles):
    st = les.les_stats_t()
    assert libles.les_step(None, 1, ctypes.byref(st)) == les.LES_EINVAL
    assert libles.les_get_fields(None, None, None, None, None) == les.LES_EINVAL


def test_header_constants_match_binding():
    """Every integer #define of include/les.h that the Python binding also
    names has the same value there."""
    txt = open(os.path.join(ROOT, "include", "les.h")).read()
    pat = r"^#define\s+(LES_\w+)\s+\(?(-?\d+)\)?\s*(?:/\*.*\*/)?\s*$"
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(pat, txt, flags=re.M)}
    assert "LES_NET_KERNELS_LAYERS" in defs and "LES_EINVAL" in defs
    shared = [k for k in defs if hasattr(les, k)]
    assert len(shared) >= 10
    for k in shared:
        assert getattr(les, k) == defs[k], k
