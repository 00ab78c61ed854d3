"""The allocation-free residual entry point, for callers that cannot call
cudaMalloc (code inside another framework's memory pool, programs with a
device-memory budget fixed at start-up, callers that must not allocate while
a stream capture is in progress).  les_residual_noalloc keeps its scratch in
a fixed device array of the library; its norms must equal the ones the
handle path reports for the same pressure and right-hand side
(les_pressure_solve), on two calls in a row, for FP64 and FP32 arrays, on
periodic axes, and on a grid large enough that its 4096 blocks stride over
several cells each.  On the small grids the norms are also checked against
the FP64 oracle's residual of the same pressure.

This file is collected last on purpose, so a failure here does not hide the
results of the other GPU tests."""

import ctypes

import numpy as np
import pytest

from oracle.oracle import Oracle, A_P, A_RHS
from paper_1504_02264_gb300 import scene

pytestmark = pytest.mark.gpu

les = pytest.importorskip("paper_1504_02264_gb300.les")


def case_scene(case):
    if case == "large":
        nx, ny, nz = 128, 96, 96           # 1.18 M cells > 4096 blocks x 256 threads
    else:
        nx, ny, nz = 40, 24, 12
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:5, 6:12, 8:14] = 1
    solid[:3, 14:20, 22:26] = 1
    if case == "periodic":
        return scene.box_scene(nx, ny, nz, dz=np.full(nz, 2.0), solid=solid,
                               bc=(scene.BC_INOUT, scene.BC_PERIODIC, scene.BC_PERIODIC),
                               fixed_sweeps=1, max_sweeps=25)
    return scene.box_scene(nx, ny, nz, dz=scene.stretched_dz(nz), solid=solid, fixed_sweeps=1, max_sweeps=25)


@pytest.mark.parametrize("case,prec", [("wall", "fp64"), ("wall", "fp32"), ("periodic", "fp64"),
                                       ("periodic", "fp32"), ("large", "fp32")])
def test_noalloc_residual_matches_pressure_solve_twice(case, prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = case_scene(case)
    nx, ny, nz = sc.nx, sc.ny, sc.nz
    p_ = les.LES_FP64 if prec == "fp64" else les.LES_FP32
    d = les.Domain(sc, precision=p_)
    st = d.pressure_solve(scene.random_rhs(sc, 21))
    p = d.fields()[3]
    rhs = d.aux(les.LES_AUX_RHS)           # the mean-removed right-hand side the solve used
    d.close()
    dev = torch.device("cuda", 0)
    tp = torch.from_numpy(np.ascontiguousarray(p)).to(dev)
    tr = torch.from_numpy(np.ascontiguousarray(rhs)).to(dev)
    ts = torch.from_numpy(np.ascontiguousarray(sc.solid)).to(dev)
    tz = torch.from_numpy(np.ascontiguousarray(sc.dz)).to(dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    dz = np.ascontiguousarray(sc.dz)
    g = les.les_grid_t(nx=nx, ny=ny, nz=nz, bc_x=sc.bc_x, bc_y=sc.bc_y, bc_z=sc.bc_z, dx=sc.dx, dy=sc.dy,
                       dz=dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), precision=p_)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    # the handle reports the FP64 norms of its FP64 pressure; the arrays read
    # back here are in the field type (FP32 rounds p and rhs once)
    tol = 1e-10 if prec == "fp64" else 1e-3
    for _ in range(2):                       # the shared scratch must be clean on every call
        out.zero_()
        les.les_residual_noalloc(g, tp.data_ptr(), tr.data_ptr(), ts.data_ptr(), tz.data_ptr(), out.data_ptr(),
                                 stream)
        torch.cuda.synchronize()
        res2, rhs2, rel = out.cpu().numpy()
        assert rel == pytest.approx(st["rel_residual"], rel=tol, abs=1e-300)
        assert np.sqrt(rhs2) == pytest.approx(st["rhs_norm"], rel=1e-12 if prec == "fp64" else 1e-6)
    if case != "large":
        # the FP64 oracle's residual of the same (field-type) pressure and rhs
        o = Oracle(sc)
        o.set(A_P, p.astype(np.float64))
        o.set(A_RHS, rhs.astype(np.float64))
        rel_o = o.residual()
        assert rel == pytest.approx(rel_o, rel=1e-9)
        assert np.sqrt(rhs2) == pytest.approx(o.stats()["rhs_norm"], rel=1e-12)
    big = les.les_grid_t(nx=2048, ny=2048, nz=1024, bc_x=0, bc_y=1, bc_z=2, dx=1.0, dy=1.0, precision=p_)
    with pytest.raises(les.LesError) as e:
        les.les_residual_noalloc(big, tp.data_ptr(), tr.data_ptr(), ts.data_ptr(), tz.data_ptr(), out.data_ptr(),
                                 stream)
    assert e.value.code == les.LES_EINVAL
