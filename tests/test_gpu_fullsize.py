"""GPU checks at the full size of the measured workload (the 150x150x90
random city, 100 buildings, 10% turbulent inflow) in the configuration the
benchmark times: FP32, chunked CUDA graphs, the autotuned sweep kernel, plain
and with the learned correction.  The FP64 oracle cannot run a full solve at
this size in test time, so it checks what it can compute at any size:

* the momentum phase (bondv1, les, velfg, SGS, AB2, feedbf) of one step from
  the GPU's own state, element by element (FP32 against FP64: 2e-4 of the
  velocity scale, as in the small-grid phase checks);
* the stop test: every step ends at FP64 relative residual <= 1e-6;
* the projection identity: ||div u^{n+1}|| <= 1e-6 ||div u*|| plus the
  rounding floor of FP32 face values, divergences formed by the oracle."""

import os

import numpy as np
import pytest

from oracle.oracle import Oracle, A_U, A_V, A_W, A_FU, A_FV, A_FW, A_US, A_VS, A_WS
from paper_1504_02264_gb300 import scene

pytestmark = pytest.mark.gpu

les = pytest.importorskip("paper_1504_02264_gb300.les")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    les.lib()
    yield


def workload():
    sc = scene.random_scene(seed=0)
    sc.check_every = 10
    sc.max_sweeps = 20000
    return sc


def rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300))


def divergence_check(sc, d):
    star = Oracle(sc)
    star.set(A_U, d.aux(les.LES_AUX_USTAR).astype(np.float64))
    star.set(A_V, d.aux(les.LES_AUX_VSTAR).astype(np.float64))
    star.set(A_W, d.aux(les.LES_AUX_WSTAR).astype(np.float64))
    div_star = star.divergence()
    chk = Oracle(sc)
    u, v, w, p = [a.astype(np.float64) for a in d.fields()]
    chk.set_fields(u, v, w, p)
    div = chk.divergence()
    dz = sc.dz[:, None, None]
    mag = ((np.abs(u[:, :, 1:]) + np.abs(u[:, :, :-1])) / sc.dx + (np.abs(v[:, 1:]) + np.abs(v[:, :-1])) / sc.dy +
           (np.abs(w[1:]) + np.abs(w[:-1])) / dz) * (sc.solid == 0)
    floor = 2.0 ** -24 * np.linalg.norm(mag)
    assert np.linalg.norm(div) <= 1e-6 * np.linalg.norm(div_star) + 3 * floor, \
        (np.linalg.norm(div), np.linalg.norm(div_star), floor)


@pytest.mark.parametrize("learned", [False, True])
def test_bench_workload_full_size(learned):
    sc = workload()
    d = les.Domain(sc)
    for _ in range(3):
        st = d.step()
        assert st["rc"] == 0 and st["rel_residual"] <= 1e-6
    d.autotune_sor(sweeps=10)
    net = None
    if learned:
        from paper_1504_02264_gb300 import train
        net = train.load(os.path.join(os.path.dirname(les.__file__), "weights", "warmstart.npz"))
        d.set_warmstart(net)
        d.set_net_schedule(10)
    # the oracle's momentum phase from the GPU's state before the step
    u, v, w, p = [a.astype(np.float64) for a in d.fields()]
    F = [d.aux(a).astype(np.float64) for a in (les.LES_AUX_FU, les.LES_AUX_FV, les.LES_AUX_FW)]
    step_index = d.step(0)["step"]
    o = Oracle(sc)
    o.set_fields(u, v, w, p)
    for a, arr in zip((A_FU, A_FV, A_FW), F):
        o.set(a, arr)
    o.step_index = step_index
    o.bc_fill()
    o.les_nut()
    o.momentum()
    o.outflow_fix()
    st = d.step()
    assert st["rc"] == 0 and st["rel_residual"] <= 1e-6, st
    assert st["graph"] == 1
    vel = max(np.abs(x).max() for x in (u, v, w))
    for aux, arr in ((les.LES_AUX_USTAR, A_US), (les.LES_AUX_VSTAR, A_VS), (les.LES_AUX_WSTAR, A_WS)):
        err = float(np.abs(d.aux(aux).astype(np.float64) - o.get(arr)).max()) / vel
        assert err <= 2e-4, (aux, err)
    divergence_check(sc, d)
    for _ in range(2):
        st = d.step()
        assert st["rc"] == 0 and st["rel_residual"] <= 1e-6
    divergence_check(sc, d)
    d.close()
    if net is not None:
        net.close()
