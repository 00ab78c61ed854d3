"""The allocation-free residual entry point, for callers that cannot call
cudaMalloc (code inside another framework's memory pool, programs with a
device-memory budget fixed at start-up, callers that must not allocate while
a stream capture is in progress).  les_residual_noalloc keeps its scratch in
a fixed device array of the library; its norms must equal the ones the
handle path reports for the same pressure and right-hand side.

This file is collected last on purpose, so a failure here does not hide the
results of the other GPU tests."""

import ctypes

import numpy as np
import pytest

from paper_1504_02264_gb300 import scene

pytestmark = pytest.mark.gpu

les = pytest.importorskip("paper_1504_02264_gb300.les")


def test_noalloc_residual_matches_pressure_solve_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nx, ny, nz = 40, 24, 12
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:5, 6:12, 8:14] = 1
    solid[:3, 14:20, 22:26] = 1
    sc = scene.box_scene(nx, ny, nz, dz=scene.stretched_dz(nz), solid=solid, fixed_sweeps=1, max_sweeps=25)
    d = les.Domain(sc, precision=les.LES_FP64)
    st = d.pressure_solve(scene.random_rhs(sc, 21))
    p = d.fields()[3]
    rhs = d.aux(les.LES_AUX_RHS)           # the mean-removed right-hand side the solve used
    dev = torch.device("cuda", 0)
    tp = torch.from_numpy(np.ascontiguousarray(p)).to(dev)
    tr = torch.from_numpy(np.ascontiguousarray(rhs)).to(dev)
    ts = torch.from_numpy(np.ascontiguousarray(sc.solid)).to(dev)
    tz = torch.from_numpy(np.ascontiguousarray(sc.dz)).to(dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    dz = np.ascontiguousarray(sc.dz)
    g = les.les_grid_t(nx=nx, ny=ny, nz=nz, bc_x=sc.bc_x, bc_y=sc.bc_y, bc_z=sc.bc_z, dx=sc.dx, dy=sc.dy,
                       dz=dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), precision=les.LES_FP64)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for _ in range(2):                       # the shared scratch must be clean on every call
        out.zero_()
        les.les_residual_noalloc(g, tp.data_ptr(), tr.data_ptr(), ts.data_ptr(), tz.data_ptr(), out.data_ptr(),
                                 stream)
        torch.cuda.synchronize()
        res2, rhs2, rel = out.cpu().numpy()
        assert rel == pytest.approx(st["rel_residual"], rel=1e-10, abs=1e-300)
        assert np.sqrt(rhs2) == pytest.approx(st["rhs_norm"], rel=1e-12)
    big = les.les_grid_t(nx=2048, ny=2048, nz=1024, bc_x=0, bc_y=1, bc_z=2, dx=1.0, dy=1.0, precision=les.LES_FP64)
    with pytest.raises(les.LesError) as e:
        les.les_residual_noalloc(big, tp.data_ptr(), tr.data_ptr(), ts.data_ptr(), tz.data_ptr(), out.data_ptr(),
                                 stream)
    assert e.value.code == les.LES_EINVAL
