"""Training and evaluation of the learned SOR warm start.

The network (kernels and Adam in the CUDA library) learns the map from a
Poisson residual to the correction that removes it.  Its training pairs are
generated by the plain solver: FP32 domains step forward with recording on,
and each step's solve records the residual r_k of its iterate at the first
FP64 refinement after k sweeps (k = 0 is the start of the solve) together
with the remaining correction p_solved - p_k.  Pairs with k > 0 are the
residuals the network sees when it is applied inside a solve.

    python -m paper_1504_02264_gb300.train --out weights.npy

trains on lattice runs (the 64x64x32 workload with varied seeds and building
heights) and random-city runs, then compares sweeps and time per step on a
150x150x90 random city for the previous-step start, the one-shot learned start
and the learned correction applied every m sweeps.  PyTorch only holds the
device buffers.
"""

from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import les, scene


def _require_torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("training needs a CUDA device")
    return torch


def save(net: les.Net, path: str):
    """Parameters and input stride of a trained network (.npz)."""
    np.savez(path, params=net.params(), stride=np.int32(net.stride))


def load(path: str, seed: int = 0) -> les.Net:
    z = np.load(path)
    net = les.Net(seed=seed, stride=int(z["stride"]))
    net.set_params(z["params"])
    return net


def coarse_residual_params(nparam: int) -> np.ndarray:
    """Weights under which the network computes q = r_coarse / rms: the
    non-learned coarse-grid correction that the learned one is measured
    against (same cycle, same kernels, same cost).  The first convolution
    passes the residual channel as +x and -x through its centre tap, the
    ReLU splits it into positive and negative parts, every other
    convolution is zero (the decoder adds its skips back unchanged, so the
    finest level's output is conv0's), and the head recombines the two
    parts: y = relu(x) - relu(-x) = x."""
    theta = np.zeros(nparam, np.float32)
    cin0, cout0 = 16, 16
    centre = 13                       # tap (dz, dy, dx) = (1, 1, 1)
    w0 = np.zeros((27, cout0, cin0), np.float32)
    w0[centre, 0, 0] = 1.0
    w0[centre, 1, 0] = -1.0
    theta[:w0.size] = w0.ravel()
    theta[-16] = 1.0                  # head: channel 0 minus channel 1
    theta[-15] = -1.0
    return theta


def training_scenes(n_lattice: int, n_city: int, seed: int, city_shape=(96, 96, 48), n_city2: int = 0,
                    city_shape2=(150, 150, 90)):
    """Lattice scenes (turbulent inflow for variety) and random cities of two
    sizes (seeds 1000+ and 2000+, disjoint from the evaluation and bench cities)."""
    out = []
    for s in range(n_lattice):
        sc = scene.lattice_scene(seed=seed + s)
        sc.turb, sc.fixed_sweeps, sc.tol = 0.1, 0, 1e-7
        sc.max_sweeps, sc.check_every = 60000, 20
        out.append(sc)
    for base, n, (nx, ny, nz) in ((1000, n_city, city_shape), (2000, n_city2, city_shape2)):
        for s in range(n):
            sc = scene.random_scene(seed=seed + base + s, nx=nx, ny=ny, nz=nz,
                                    n_buildings=max(8, int(100 * nx * ny / (150 * 150))),
                                    x_margin=min(16, nx // 8), tol=1e-7, max_sweeps=60000, check_every=20)
            out.append(sc)
    return out


def generate(scenes, steps: int, spinup: int, record_points, seed: int = 0, log=print, net=None, net_every=0,
             groups=None):
    """Run each scene and record one (r_k, remaining correction) pair per step.

    With `net`, the solves run with that network correction every `net_every`
    sweeps, so the recorded residuals are the ones the network meets in its
    own loop.  Returns (and extends) {shape: (R, T, M)} with R, T float32
    device tensor lists [nz, ny, nx] (residuals, targets) and M the unknown
    mask of each pair."""
    torch = _require_torch()
    rng = np.random.default_rng(seed)
    groups = {} if groups is None else groups
    for sc in scenes:
        dom = les.Domain(sc)
        dom.set_graph(True)
        for _ in range(spinup):
            dom.step()
        if net is not None:
            dom.set_warmstart(net)
            dom.set_net_schedule(net_every)
        dom.set_record(True)
        mask = torch.from_numpy(dom.aux(les.LES_AUX_MASK)).cuda()
        rs, ts = [], []
        t0 = time.time()
        sw = 0
        for _ in range(steps):
            k = int(rng.choice(record_points))
            dom.set_record(True, after_sweeps=k)
            st = dom.step()
            sw += st["sweeps"]
            if st["rc"] != 0:
                continue
            try:
                r0 = dom.aux(les.LES_AUX_R0)
            except les.LesError:
                continue                  # converged before the record point
            rs.append(torch.from_numpy(r0).cuda())
            ts.append(torch.from_numpy(dom.aux(les.LES_AUX_DELTA)).cuda())
        dom.close()
        shape = (sc.nz, sc.ny, sc.nx)
        R, T, M = groups.get(shape, ([], [], []))
        R += rs
        T += ts
        M += [mask] * len(rs)
        groups[shape] = (R, T, M)
        log(f"  {sc.name} seed {sc.seed}: {len(rs)} pairs, {sw / max(1, steps):.0f} sweeps/step, "
            f"{time.time() - t0:.1f} s")
    return groups


def stack(groups):
    torch = _require_torch()
    return {s: (torch.stack(R), torch.stack(T), torch.stack(M)) for s, (R, T, M) in groups.items()}


def train(net: les.Net, data, iters: int, batch: int, lr: float, seed: int = 0, log=print, log_every=100):
    """Adam with a cosine learning-rate decay; batches drawn from one shape group."""
    torch = _require_torch()
    rng = np.random.default_rng(seed)
    shapes = list(data)
    weights = np.array([data[s][0].shape[0] for s in shapes], np.float64)
    weights /= weights.sum()
    hist = []
    t0 = time.time()
    for it in range(iters):
        s = shapes[int(rng.choice(len(shapes), p=weights))]
        R, T, M = data[s]
        idx = torch.from_numpy(rng.integers(0, R.shape[0], batch)).cuda()
        r, t, m = R[idx].contiguous(), T[idx].contiguous(), M[idx].contiguous()
        nz, ny, nx = s
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / max(1, iters)))
        loss = les.les_net_train_step(net.h, r.data_ptr(), m.data_ptr(), t.data_ptr(), batch, nx, ny, nz,
                                      max(lr_t, 1e-3 * lr))
        hist.append(loss)
        if log_every and (it + 1) % log_every == 0:
            log(f"  iter {it + 1}: loss {np.mean(hist[-log_every:]):.4f} ({time.time() - t0:.0f} s)")
    return hist


def evaluate(net: les.Net | None, sc, steps: int, spinup: int, schedules=(0,), log=print, persistent=False,
             start=True):
    """Sweeps and milliseconds per step to the scene's tolerance for the
    previous-step start and, with a network, for each correction schedule
    (0 = one-shot warm start; m > 0 = also every m sweeps).  All runs start
    from the same spun-up state; the network's own time is included."""
    torch = _require_torch()
    base = les.Domain(sc)
    for _ in range(spinup):
        base.step()
    state = base.get_state()
    (tile, kc), _ = base.autotune_sor(sweeps=20)
    base.close()
    modes = [("prev", None)] + ([(f"net_every_{m}", m) for m in schedules] if net is not None else [])
    res = {}
    for name, m in modes:
        dom = les.Domain(sc)
        dom.set_state(state)
        dom.set_sor_config(tile, kc)
        if m is not None:
            dom.set_warmstart(net)
            dom.set_net_schedule(m)
            dom.set_net_kernels(persistent)
            dom.set_net_start(start)
        sweeps, ms, ok = [], [], True
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = dom.step()
            torch.cuda.synchronize()
            ms.append(1e3 * (time.perf_counter() - t0))
            sweeps.append(st["sweeps"])
            ok &= st["rc"] == 0 and st["rel_residual"] <= sc.tol
        dom.close()
        res[name] = {"sweeps_per_step": float(np.mean(sweeps)), "ms_per_step": float(np.mean(ms)),
                     "converged": bool(ok), "sor_tile": [tile, kc]}
        log(f"  {name}: {res[name]}")
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default="warmstart.npz")
    ap.add_argument("--init", default=None, help="start from this network (.npz)")
    ap.add_argument("--stride", default="4", help="input stride(s) of the network, e.g. 2,4 (one net each)")
    ap.add_argument("--city-size", default="96x96x48")
    ap.add_argument("--cities2", type=int, default=0, help="random-city scenes of the second size")
    ap.add_argument("--city-size2", default="150x150x90")
    ap.add_argument("--lattice", type=int, default=16, help="lattice scenes (seeds)")
    ap.add_argument("--cities", type=int, default=8, help="random-city scenes")
    ap.add_argument("--steps", type=int, default=40, help="recorded steps per scene")
    ap.add_argument("--spinup", type=int, default=5)
    ap.add_argument("--record-points", default="0,40,100,200,400,800")
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--eval-steps", type=int, default=4)
    ap.add_argument("--eval-spinup", type=int, default=8)
    ap.add_argument("--eval-size", default="150x150x90")
    ap.add_argument("--schedules", default="0,50,100,200")
    ap.add_argument("--json", default=None, help="write the evaluation here")
    ap.add_argument("--eval-only", default=None, help="evaluate these trained networks (.npz, comma separated)")
    ap.add_argument("--persistent", action="store_true", help="evaluate with the persistent coarse network")
    ap.add_argument("--no-start", action="store_true", help="no network correction at the start of a solve")
    ap.add_argument("--dagger", default=None, help="also record pairs with this network in the loop (.npz)")
    ap.add_argument("--dagger-every", type=int, default=10)
    ap.add_argument("--dagger-points", default="0,10,20,30,50,80,120,200")
    a = ap.parse_args(argv)
    les.lib()
    if a.eval_only:
        nx, ny, nz = (int(x) for x in a.eval_size.split("x"))
        ev_sc = scene.random_scene(seed=a.seed + 7777, nx=nx, ny=ny, nz=nz, max_sweeps=60000, check_every=20)
        report = {"eval_scene": ev_sc.name, "nets": {}}
        for path in a.eval_only.split(","):
            net = load(path)
            print(f"{path} (stride {net.stride}) on {ev_sc.name} seed {ev_sc.seed}:", flush=True)
            report["nets"][path] = evaluate(net, ev_sc, a.eval_steps, a.eval_spinup,
                                            [int(x) for x in a.schedules.split(",")],
                                            persistent=a.persistent, start=not a.no_start)
            net.close()
        print(json.dumps(report), flush=True)
        if a.json:
            with open(a.json, "w") as f:
                json.dump(report, f, indent=1)
        return
    t0 = time.time()
    pts = [int(x) for x in a.record_points.split(",")]
    print(f"generating pairs: {a.lattice} lattice + {a.cities} city scenes x {a.steps} steps", flush=True)
    cs = tuple(int(x) for x in a.city_size.split("x"))
    cs2 = tuple(int(x) for x in a.city_size2.split("x"))
    scenes = training_scenes(a.lattice, a.cities, a.seed, cs, a.cities2, cs2)
    groups = generate(scenes, a.steps, a.spinup, pts, a.seed)
    if a.dagger:
        # pairs from solves that run with a network in the loop
        dnet = load(a.dagger)
        dpts = [int(x) for x in a.dagger_points.split(",")]
        print(f"pairs with {a.dagger} every {a.dagger_every} sweeps in the loop", flush=True)
        generate(scenes, a.steps, a.spinup, dpts, a.seed + 1, net=dnet, net_every=a.dagger_every, groups=groups)
        dnet.close()
    data = stack(groups)
    npairs = sum(v[0].shape[0] for v in data.values())
    print(f"{npairs} pairs in {time.time() - t0:.0f} s", flush=True)
    nx, ny, nz = (int(x) for x in a.eval_size.split("x"))
    ev_sc = scene.random_scene(seed=a.seed + 7777, nx=nx, ny=ny, nz=nz, max_sweeps=60000, check_every=20)
    report = {"pairs": npairs, "iters": a.iters, "eval_scene": ev_sc.name, "nets": {}}
    for st in (int(x) for x in a.stride.split(",")):
        net = load(a.init, a.seed) if a.init else les.Net(seed=a.seed)
        net.stride = st
        hist = train(net, data, a.iters, a.batch, a.lr, a.seed)
        out = a.out if "," not in a.stride else a.out.replace(".npz", f"_s{st}.npz")
        save(net, out)
        print(f"stride {st}: trained {a.iters} iterations, final loss {np.mean(hist[-100:]):.4f}; saved {out}",
              flush=True)
        print(f"evaluation on {ev_sc.name} seed {ev_sc.seed}:", flush=True)
        res = evaluate(net, ev_sc, a.eval_steps, a.eval_spinup, [int(x) for x in a.schedules.split(",")])
        report["nets"][st] = {"final_loss": float(np.mean(hist[-100:])), "loss_first": float(np.mean(hist[:100])),
                              "file": out, "eval": res}
        net.close()
    print(json.dumps(report), flush=True)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()
