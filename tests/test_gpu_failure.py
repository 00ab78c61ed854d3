"""Failure detection on the GPU without a fault: a bounded device wait whose
transaction never arrives must give up, report LES_ETIMEOUT to the host, and
leave the CUDA context usable."""

import time

import numpy as np
import pytest

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


def test_bounded_wait_times_out_and_context_survives():
    t0 = time.perf_counter()
    rc = les.les_selftest_wait_timeout(2_000_000)           # 2 ms limit
    assert rc == les.LES_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert b"expected" in les.lib().les_last_error(None)
    # the context still runs ordinary work
    sc = scene.lattice_scene(0, nx=32, ny=32, nz=16)
    d = les.Domain(sc)
    st = d.step(2)
    assert st["rc"] == 0 and np.all(np.isfinite(d.fields()[0]))
    d.close()


def test_selftest_rejects_bad_limits():
    with pytest.raises(les.LesError):
        les.les_selftest_wait_timeout(10)
