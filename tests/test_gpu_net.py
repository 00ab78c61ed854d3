"""GPU tests of the learned SOR warm start: the BF16 tensor-core network
against the FP64 NumPy network oracle (forward and gradient), its training
step, the recording of training pairs, and the warm start inside the solver.

Tolerances.  The GPU network stores activations and activation gradients in
BF16 (unit roundoff u = 2^-9) and accumulates in FP32.  The longest forward
chain rounds about 14 times (input, 7 convolution outputs, 3 pools, 3 skip
sums), so the worst-case relative error is ~14u = 2.7% and the random-walk
estimate sqrt(14)u = 0.7%; the forward bar is 2% in relative L2 norm.  The
backward pass adds about as many roundings again: 5% per layer gradient, with
the direction (cosine) within 0.998.  The oracle uses the same BF16-rounded
convolution weights, so weight rounding is not part of the comparison."""

import numpy as np
import pytest

from oracle import net_oracle
from oracle.oracle import Oracle
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


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), kept as float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def oracle_theta(theta32):
    """The parameters the GPU computes with: BF16 convolution weights, FP32 head."""
    t = theta32.astype(np.float32).copy()
    nh = net_oracle.HEAD
    t[:-nh] = bf16_round(t[:-nh])
    return t.astype(np.float64)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def sample(rng, shape, fluid=0.8):
    r = rng.standard_normal(shape)
    # smooth-ish residual plus noise, like an SOR residual
    mask = (rng.random(shape) < fluid).astype(np.float64)
    return r * mask, mask


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.fixture()
def net():
    n = les.Net(seed=11)
    yield n
    torch.cuda.synchronize()
    n.close()


def test_engine_setting(net):
    assert net.engine == les.LES_NET_TCGEN05            # the default
    net.engine = les.LES_NET_MMA_SYNC
    assert net.engine == les.LES_NET_MMA_SYNC
    net.engine = les.LES_NET_TCGEN05_GMEM_SPLIT
    assert net.engine == les.LES_NET_TCGEN05_GMEM_SPLIT
    with pytest.raises(les.LesError):
        net.engine = 7


def test_stride_setting(net):
    assert net.stride == 1
    net.stride = 4
    assert net.stride == 4
    with pytest.raises(les.LesError):
        net.stride = 3


def test_param_count_and_roundtrip(net):
    ws = [27 * ci * co for ci, co in zip(net_oracle.CIN, net_oracle.COUT)]
    assert net.nparam == sum(ws) + net_oracle.HEAD
    theta = net_oracle.init_params(5).astype(np.float32)
    net.set_params(theta)
    assert np.array_equal(net.params(), theta)
    assert np.all(np.isfinite(net.params()))


@pytest.mark.parametrize("engine", ["tcgen05", "mma.sync"])
@pytest.mark.parametrize("shape,stride", [((7, 11, 37), 1), ((1, 1, 1), 1), ((5, 9, 16), 1), ((3, 4, 17), 1),
                                          ((13, 22, 70), 2), ((17, 30, 61), 4), ((3, 5, 6), 4), ((9, 40, 19), 1)])
def test_forward_matches_oracle(net, shape, stride, engine):
    """(nz, ny, nx) = 7x11x37 spans 3x3x4 tiles with ragged tails on every
    level; the strided cases pool to ragged coarse grids and prolongate back;
    9x40x19 spans several 8x16 tiles of the tcgen05 kernel with ragged tails.
    Both tensor-core engines (tcgen05 and warp-level mma.sync)."""
    rng = np.random.default_rng(sum(shape))
    theta = net_oracle.init_params(7).astype(np.float32)
    net.set_params(theta)
    net.stride = stride
    net.engine = les.LES_NET_TCGEN05 if engine == "tcgen05" else les.LES_NET_MMA_SYNC
    r, mask = sample(rng, shape)
    if mask.sum() == 0:
        mask.flat[0] = 1.0
    y = torch.empty(shape, dtype=torch.float32, device="cuda")
    dr, dm = dev(r), dev(mask)
    nz, ny, nx = shape
    les.les_net_forward(net.h, dr.data_ptr(), dm.data_ptr(), y.data_ptr(), nx, ny, nz)
    yg = y.cpu().numpy().astype(np.float64)
    yo = net_oracle.forward_strided(oracle_theta(theta), r.astype(np.float32).astype(np.float64), mask, stride)
    assert np.all(yg[mask == 0] == 0.0)
    err = rel_l2(yg, yo)
    assert err <= 2e-2, err
    assert np.abs(yg - yo).max() <= 5e-2 * np.abs(yo).max()


def test_forward_scale_invariant(net):
    """The input is normalised by its RMS: r and 2r give bit-identical outputs."""
    rng = np.random.default_rng(1)
    shape = (6, 10, 20)
    r, mask = sample(rng, shape)
    nz, ny, nx = shape
    ys = []
    for s in (1.0, 2.0):
        y = torch.empty(shape, dtype=torch.float32, device="cuda")
        dr, dm = dev(r * s), dev(mask)
        les.les_net_forward(net.h, dr.data_ptr(), dm.data_ptr(), y.data_ptr(), nx, ny, nz)
        ys.append(y.cpu().numpy())
    assert np.array_equal(ys[0], ys[1])


@pytest.mark.parametrize("engine", ["tcgen05", "mma.sync"])
@pytest.mark.parametrize("shape,stride", [((5, 9, 21), 1), ((10, 17, 40), 2)])
def test_gradient_matches_oracle(net, shape, stride, engine):
    rng = np.random.default_rng(2)
    B = 2
    theta = net_oracle.init_params(9).astype(np.float32)
    net.set_params(theta)
    net.stride = stride
    net.engine = les.LES_NET_TCGEN05 if engine == "tcgen05" else les.LES_NET_MMA_SYNC
    rs, ms, ts = [], [], []
    for _ in range(B):
        r, m = sample(rng, shape)
        t = rng.standard_normal(shape) * m
        rs.append(r.astype(np.float32)); ms.append(m); ts.append(t.astype(np.float32))
    nz, ny, nx = shape
    dr, dm, dt = dev(np.stack(rs)), dev(np.stack(ms)), dev(np.stack(ts))
    g = torch.empty(net.nparam, dtype=torch.float32, device="cuda")
    L = les.les_net_gradient(net.h, dr.data_ptr(), dm.data_ptr(), dt.data_ptr(), B, nx, ny, nz, g.data_ptr())
    Lo, go = net_oracle.loss_and_grad_strided(oracle_theta(theta), [x.astype(np.float64) for x in rs], ms,
                                              [x.astype(np.float64) for x in ts], stride)
    assert abs(L - Lo) <= 2e-2 * abs(Lo), (L, Lo)
    gg = g.cpu().numpy().astype(np.float64)
    o = 0
    for k, (ci, co) in enumerate(zip(net_oracle.CIN, net_oracle.COUT)):
        n = 27 * ci * co
        a, b = gg[o:o + n], go[o:o + n]
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert rel_l2(a, b) <= 5e-2 and cos >= 0.998, (k, rel_l2(a, b), cos)
        o += n
    assert rel_l2(gg[o:], go[o:]) <= 5e-2


def test_train_step_reduces_loss(net):
    rng = np.random.default_rng(3)
    shape, B = (8, 12, 24), 4
    nz, ny, nx = shape
    rs, ms, ts = [], [], []
    for _ in range(B):
        m = (rng.random(shape) < 0.85).astype(np.float32)
        t = rng.standard_normal(shape).astype(np.float32)
        # a target the network can fit: a smoothed version of the input
        r = t.copy()
        for ax in range(3):
            r = 0.5 * r + 0.25 * (np.roll(r, 1, ax) + np.roll(r, -1, ax))
        rs.append(r * m); ms.append(m); ts.append(t * m)
    dr, dm, dt = dev(np.stack(rs)), dev(np.stack(ms)), dev(np.stack(ts))
    losses = [les.les_net_train_step(net.h, dr.data_ptr(), dm.data_ptr(), dt.data_ptr(), B, nx, ny, nz, 1e-3)
              for _ in range(40)]
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.8 * losses[0], losses[::8]


def city(nx=48, ny=32, nz=16, seed=4, bc=(scene.BC_INOUT, scene.BC_FREESLIP, scene.BC_WALL), **kw):
    """A small FP32 city: five blocks, turbulent inflow, solves to tolerance."""
    kw.setdefault("fixed_sweeps", 0)
    rng = np.random.default_rng(seed)
    solid = np.zeros((nz, ny, nx), np.uint8)
    for _ in range(5):
        x0 = int(rng.integers(8, nx - 12))
        y0 = int(rng.integers(1, ny - 7))
        h = int(rng.integers(3, nz - 3))
        solid[:h, y0:y0 + 6, x0:x0 + 6] = 1
    return scene.box_scene(nx, ny, nz, dz=scene.stretched_dz(nz), solid=solid, bc=bc, turb=0.1, seed=seed,
                           **kw)


def test_recorded_pair_solves_the_system():
    """The recorded correction delta of a converged solve satisfies A delta = r0
    to the solve's tolerance (FP64 grid, checked with the oracle's operator)."""
    sc = city(tol=1e-8, max_sweeps=40000, check_every=20)
    dom = les.Domain(sc, precision=les.LES_FP64)
    dom.set_record(True)
    for _ in range(3):
        st = dom.step()
        assert st["rc"] == 0 and st["rel_residual"] <= 1e-8
    r0 = dom.aux(les.LES_AUX_R0)
    delta = dom.aux(les.LES_AUX_DELTA)
    mask = dom.aux(les.LES_AUX_MASK)
    o = Oracle(sc)
    Ad = o.apply_A(delta)
    assert np.all(delta[mask == 0] == 0) and np.all(r0[mask == 0] == 0)
    err = np.linalg.norm((Ad - r0)[mask == 1])
    assert err <= 1.01e-8 * st["rhs_norm"] + 1e-12 * np.linalg.norm(r0), (err, st["rhs_norm"])
    assert np.linalg.norm(r0) > 10 * err          # the pair is not trivial
    dom.close()


def energy(o, sc, e):
    """Error energy -e^T V A e with V = diag(dz_k) (V A is symmetric), over the unknowns."""
    Ae = o.apply_A(e)
    return float(-np.sum(np.asarray(sc.dz)[:, None, None] * e * Ae))


def test_warm_start_line_search_lowers_error_energy(net):
    """From p = 0 on a random right-hand side, the learned start p0 = alpha q
    is no further from the exact solution (oracle, FP64, 1e-12) in the energy
    norm than p = 0, and the solve still reaches its tolerance."""
    sc = city(tol=1e-6, max_sweeps=40000, check_every=20)
    rhs = scene.random_rhs(sc, 5)
    dom = les.Domain(sc)
    dom.set_warmstart(net)
    dom.set_record(True)
    u, v, w, _ = dom.fields()
    dom.set_fields(u, v, w, np.zeros((sc.nz, sc.ny, sc.nx)))
    st = dom.pressure_solve(rhs)
    assert st["rc"] == 0 and st["rel_residual"] <= 1e-6
    delta = dom.aux(les.LES_AUX_DELTA).astype(np.float64)
    p_fin = dom.fields()[3].astype(np.float64)
    mask = dom.aux(les.LES_AUX_MASK)
    dom.close()
    o = Oracle(sc, tol=1e-12, max_sweeps=400000, check_every=50, fixed_sweeps=0)
    o.set_fields(*o.fields()[:3], np.zeros((sc.nz, sc.ny, sc.nx)))
    o.pressure_solve(rhs)
    assert o.stats()["rel_residual"] <= 1e-12
    p_star = o.fields()[3]
    p0 = (p_fin - delta) * mask            # the learned start (up to a constant)
    e_zero, e_net = energy(o, sc, p_star * mask), energy(o, sc, (p_star - p0) * mask)
    assert e_net <= e_zero * (1 + 1e-6), (e_net, e_zero)


def test_warm_start_schedules_converge(net):
    """Previous-step, cold and learned starts (one-shot and every 100 sweeps)
    all end every step at the same tolerance; pairs recorded after k sweeps
    are complete or reported missing."""
    sc = city(tol=1e-6, max_sweeps=40000, check_every=20)
    doms = {m: les.Domain(sc) for m in ("prev", "zero", "net", "net100")}
    doms["zero"].set_warmstart(mode=les.LES_WARM_ZERO)
    doms["net"].set_warmstart(net)
    doms["net100"].set_warmstart(net)
    doms["net100"].set_net_schedule(100)
    doms["prev"].set_record(True, after_sweeps=60)
    sweeps = {m: [] for m in doms}
    for _ in range(3):
        for m, d in doms.items():
            st = d.step()
            assert st["rc"] == 0 and st["rel_residual"] <= 1e-6, (m, st)
            sweeps[m].append(st["sweeps"])
    print("sweeps per step", sweeps)
    r = doms["prev"].aux(les.LES_AUX_R0)
    dl = doms["prev"].aux(les.LES_AUX_DELTA)
    assert np.linalg.norm(r) > 0 and np.linalg.norm(dl) > 0
    # a record point beyond the solve: no pair
    doms["prev"].set_record(True, after_sweeps=10 ** 6)
    doms["prev"].step()
    with pytest.raises(les.LesError):
        doms["prev"].aux(les.LES_AUX_R0)
    for d in doms.values():
        d.close()


@pytest.mark.parametrize("stride", [1, 4])
def test_net_cycle_graph_matches_host_loop(net, stride):
    """The network correction every 20 sweeps captured in the chunk graphs
    (device-side early exit) runs exactly the host loop's kernels: identical
    sweeps and bit-identical fields."""
    net.stride = stride
    sc = city(tol=1e-6, max_sweeps=40000, check_every=20)
    doms = []
    for graph in (True, False):
        d = les.Domain(sc)
        d.set_graph(graph)
        d.set_warmstart(net)
        d.set_net_schedule(20)
        doms.append(d)
    for _ in range(2):
        a, b = doms[0].step(), doms[1].step()
        assert a["graph"] == 1 and b["graph"] == 0
        assert a["rc"] == b["rc"] == 0 and a["sweeps"] == b["sweeps"], (a, b)
    for fa, fb in zip(doms[0].fields(), doms[1].fields()):
        assert np.array_equal(fa, fb)
    for d in doms:
        d.close()


def test_persistent_and_layer_kernels_agree(net):
    """The one-launch network correction and the per-layer launches compute
    the same correction (up to summation order): both converge every step with
    sweep counts within a few batches of each other."""
    net.stride = 4
    sc = city(tol=1e-6, max_sweeps=40000, check_every=20)
    out = {}
    for persistent in (True, False):
        d = les.Domain(sc)
        d.set_warmstart(net)
        d.set_net_schedule(20)
        d.set_net_kernels(persistent)
        sw = []
        for _ in range(3):
            st = d.step()
            assert st["rc"] == 0 and st["rel_residual"] <= 1e-6
            sw.append(st["sweeps"])
        out[persistent] = (sw, d.fields()[0])
        d.close()
    for a, b in zip(out[True][0], out[False][0]):
        assert abs(a - b) <= 60, out
    u1, u2 = out[True][1], out[False][1]
    assert np.abs(u1 - u2).max() <= 1e-3 * np.abs(u2).max()


@pytest.mark.parametrize("stride,engine,periodic", [(8, "tcgen05", True), (4, "tcgen05", False),
                                                    (2, "mma.sync", True), (1, "tcgen05", True)])
def test_folded_kernels_match_standalone(net, stride, engine, periodic):
    """The folded kernel layout (packing inside the first convolution, head
    inside the last, prolongation inside the line search) computes the values
    of the stand-alone packing, head and prolongation kernels: identical
    sweep counts and bit-identical fields after learned-mode steps in the
    graph loop, with the correction at the start of each solve and every 10
    sweeps.  Periodic x and y put wrapped cells in the line search's halo."""
    net.stride = stride
    net.engine = les.LES_NET_TCGEN05 if engine == "tcgen05" else les.LES_NET_MMA_SYNC
    kw = dict(tol=1e-6, max_sweeps=40000, check_every=10)
    if periodic:
        kw["bc"] = (scene.BC_PERIODIC, scene.BC_PERIODIC, scene.BC_WALL)
    sc = city(**kw)
    doms = []
    for mode in (les.LES_NET_KERNELS_FOLDED, les.LES_NET_KERNELS_LAYERS):
        d = les.Domain(sc)
        d.set_warmstart(net)
        d.set_net_schedule(10)
        d.set_net_kernels(mode)
        doms.append(d)
    try:
        for _ in range(2):
            a, b = doms[0].step(), doms[1].step()
            assert a["rc"] == b["rc"] == 0 and a["sweeps"] == b["sweeps"], (a, b)
        for fa, fb in zip(doms[0].fields(), doms[1].fields()):
            assert np.array_equal(fa, fb)
        print(f"stride {stride} {engine} periodic={periodic}: {a['sweeps']} sweeps, bit-identical")
    finally:
        for d in doms:
            d.close()


@pytest.mark.parametrize("stride", [8, 4])
def test_estimate_pooling_matches_pooling_kernel(net, stride):
    """On an FP32 grid with no periodic axis the estimate before each network
    correction also pools the residual and the mask (in the pooling kernel's
    order) and forms the RMS, and the correction skips its pooling kernel;
    LES_NET_KERNELS_OWN_POOL keeps that kernel.  The pooled input is the same,
    and the RMS (FP64, summed in another block order) gives the same FP32
    scale here: identical sweep counts and bit-identical fields after
    learned-mode steps in the graph loop, with fewer launches."""
    net.stride = stride
    sc = city(tol=1e-6, max_sweeps=40000, check_every=10)
    out = []
    for mode in (les.LES_NET_KERNELS_FOLDED, les.LES_NET_KERNELS_FOLDED | les.LES_NET_KERNELS_OWN_POOL):
        d = les.Domain(sc)
        try:
            d.set_warmstart(net)
            d.set_net_schedule(10)
            d.set_net_kernels(mode)
            sts = [d.step() for _ in range(2)]
            assert all(st["rc"] == 0 and st["graph"] == 1 for st in sts), sts
            out.append(([st["sweeps"] for st in sts], sts[-1]["launches"], d.fields()))
        finally:
            d.close()
    assert out[0][0] == out[1][0], (out[0][0], out[1][0])
    assert out[0][1] < out[1][1], (out[0][1], out[1][1])
    for a, b in zip(out[0][2], out[1][2]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("stride", [8, 4])
def test_cluster_split_matches_global_split(net, stride):
    """The small layers split their input channels over CTAs; the tcgen05
    engine adds the partial sums over distributed shared memory in a
    thread-block cluster, LES_NET_TCGEN05_GMEM_SPLIT through global memory,
    both in the order of the split.  At stride 8 on this city the coarse grid
    is 6x4x2 and the splits reach 8 CTAs.  Identical sweep counts and
    bit-identical fields after learned-mode steps."""
    net.stride = stride
    sc = city(tol=1e-6, max_sweeps=40000, check_every=10)
    out = []
    for engine in (les.LES_NET_TCGEN05, les.LES_NET_TCGEN05_GMEM_SPLIT):
        net.engine = engine
        d = les.Domain(sc)
        try:
            d.set_warmstart(net)
            d.set_net_schedule(10)
            sw = [d.step()["sweeps"] for _ in range(2)]
            out.append((sw, d.fields()))
        finally:
            d.close()
    assert out[0][0] == out[1][0], (out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)


def test_warm_start_rejects_bad_use(net):
    sc = city()
    d64 = les.Domain(sc, precision=les.LES_FP64)
    with pytest.raises(les.LesError):
        d64.set_warmstart(net)
    d32 = les.Domain(sc)
    with pytest.raises(les.LesError):
        d32.aux(les.LES_AUX_R0)                 # recording is off
    with pytest.raises(les.LesError):
        les.les_set_warmstart(d32.h, 7, None)
    with pytest.raises(les.LesError):
        d32.set_net_kernels(3)                  # no such kernel layout
    d64.close()
    d32.close()


def test_trained_network_gain():
    """What the trained network (the package's weights) gains on an unseen
    random city, the same tolerance every step, network time included:
    against plain SOR, and against the same correction cycle (every 10
    sweeps, stride 8, energy-norm step) run with untrained He-normal weights
    and with the non-learned coarse correction q = prolongated pooled
    residual (train.coarse_residual_params).  The last two separate what
    the training buys from what the coarse-correction structure gives."""
    import os
    import time
    from paper_1504_02264_gb300 import train
    path = os.path.join(os.path.dirname(les.__file__), "weights", "warmstart.npz")
    nets = {"trained": train.load(path), "untrained": les.Net(seed=123, stride=8)}
    nets["coarse_residual"] = les.Net(seed=0, stride=8)
    nets["coarse_residual"].set_params(train.coarse_residual_params(nets["coarse_residual"].nparam))
    sc = scene.random_scene(seed=4242, nx=96, ny=96, nz=48, n_buildings=40, x_margin=12, max_sweeps=60000,
                            check_every=20)
    base = les.Domain(sc)
    for _ in range(4):
        base.step()
    state = base.get_state()
    base.close()
    res = {}
    for mode in ("plain", "trained", "untrained", "coarse_residual"):
        d = les.Domain(sc)
        d.set_state(state)
        if mode != "plain":
            d.set_warmstart(nets[mode])
            d.set_net_schedule(10)
            d.step()                      # builds its graphs
            d.set_state(state)
        sw, ms = [], []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = d.step()
            torch.cuda.synchronize()
            ms.append(1e3 * (time.perf_counter() - t0))
            assert st["rc"] == 0 and st["rel_residual"] <= 1e-6, (mode, st)
            sw.append(st["sweeps"])
        res[mode] = (float(np.mean(sw)), float(np.median(ms)))
        d.close()
    for n in nets.values():
        n.close()
    print("sweeps and ms per step:", res)
    assert res["trained"][0] * 3 <= res["plain"][0], res
    assert res["trained"][1] < res["plain"][1], res
    # what training buys over the same cycle without it
    assert res["trained"][0] < res["untrained"][0], res
    assert res["trained"][0] < res["coarse_residual"][0], res


def test_overlapped_correction_converges():
    """The network prediction overlapped with the next batch of sweeps
    (les_set_net_async): every step still ends at the tolerance, the sweeps
    stay within a third of the in-place correction's, and the fields agree
    with the in-place run to the accuracy both solves are held to."""
    import os
    import time
    from paper_1504_02264_gb300 import train
    net = train.load(os.path.join(os.path.dirname(les.__file__), "weights", "warmstart.npz"))
    sc = scene.random_scene(seed=4242, nx=96, ny=96, nz=48, n_buildings=40, x_margin=12, max_sweeps=60000,
                            check_every=20)
    base = les.Domain(sc)
    for _ in range(4):
        base.step()
    state = base.get_state()
    base.close()
    out = {}
    for mode in ("in_place", "overlapped"):
        d = les.Domain(sc)
        d.set_state(state)
        d.set_warmstart(net)
        d.set_net_schedule(10)
        d.set_net_async(mode == "overlapped")
        d.step()
        d.set_state(state)
        sw, ms = [], []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = d.step()
            torch.cuda.synchronize()
            ms.append(1e3 * (time.perf_counter() - t0))
            assert st["rc"] == 0 and st["rel_residual"] <= 1e-6 and st["graph"] == 1, (mode, st)
            sw.append(st["sweeps"])
        out[mode] = (sw, float(np.median(ms)), d.fields())
        d.close()
    net.close()
    print("in-place vs overlapped (sweeps, ms per step):", out["in_place"][:2], out["overlapped"][:2])
    assert sum(out["overlapped"][0]) <= 1.34 * sum(out["in_place"][0])
    vel = max(np.abs(a).max() for a in out["in_place"][2][:3])
    err = max(np.abs(a.astype(np.float64) - b).max() for a, b in zip(out["overlapped"][2][:3], out["in_place"][2][:3]))
    assert err <= 1e-4 * vel
