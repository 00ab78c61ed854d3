"""Profiling driver: run LES steps through the C ABI only (no torch), so that
an external profiler sees nothing but this library's kernels.

    python -m paper_1504_02264_gb300.profile --workload random --warmup 3 --steps 2 [--range]

--range brackets the measured steps with cudaProfilerStart/Stop (for
``ncu --profile-from-start off``).  Prints one JSON line with host wall time
per step and the solver statistics.
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import les, scene


def run_ensemble(a):
    """Batched ensemble of uneven random cities (96^2-256^2 x 64-128)."""
    scs = scene.ensemble_scenes(seed=a.seed, n=a.members)
    for sc in scs:
        sc.max_sweeps = a.max_sweeps
    cells = sum(sc.ncells for sc in scs)
    ens = les.Ensemble(scs, stream=None)
    ens.set_graph(bool(a.graph))
    net = None
    if a.net:
        z = np.load(a.net)
        net = les.Net(seed=0, stream=None, stride=int(z["stride"]))
        net.set_params(z["params"])
        ens.set_warmstart(net, a.net_every)
    for _ in range(a.warmup):
        ens.step(1)
    tune = ens.autotune(sweeps=10) if a.autotune else None
    if a.ens_tile is not None:
        ens.set_tile(a.ens_tile, 4)
    if a.persistent:
        ens.set_persistent(True)
    if a.range:
        les.les_profiler_range(1)
    t0 = time.perf_counter()
    sweeps, worst, rcs = [], 0.0, []
    for _ in range(a.steps):
        st = ens.step(1)
        sweeps.append([s["sweeps"] for s in st])
        worst = max(worst, max(s["rel_residual"] for s in st))
        rcs.append(st[0]["rc"])
    t1 = time.perf_counter()
    if a.range:
        les.les_profiler_range(0)
    ms = (t1 - t0) * 1e3 / a.steps
    print(json.dumps({"workload": "ensemble", "members": a.members, "cells": cells, "steps": a.steps,
                      "ms_per_step": ms, "mcell_steps_per_s": cells / (ms * 1e-3) / 1e6,
                      "max_sweeps_per_step": [max(x) for x in sweeps],
                      "mean_member_sweeps": [sum(x) / len(x) for x in sweeps], "max_rel_residual": worst,
                      "rc": rcs, "tile": ens.tile(), "autotune": tune, "graph": a.graph, "net": a.net,
                      "persistent": a.persistent, "launches": ens.launches(),
                      "net_every": a.net_every if a.net else None,
                      "shapes": [[sc.nx, sc.ny, sc.nz] for sc in scs]}))
    ens.close()


def run_engines(a):
    """The learned step (network every --net-every sweeps) and one network
    forward on the workload's residual, per convolution engine (tcgen05 with
    the split partials added in a cluster or through global memory, and the
    warp-level mma.sync kernel; the two tcgen05 rows run twice, interleaved):
    host wall time per step, CUDA events around the forward."""
    import torch
    sc = make(a.workload, a.seed)
    z = np.load(a.net)
    out = {"workload": a.workload, "cells": sc.ncells, "rows": []}
    engines = (("tcgen05", les.LES_NET_TCGEN05), ("tcgen05 gmem split", les.LES_NET_TCGEN05_GMEM_SPLIT),
               ("mma.sync", les.LES_NET_MMA_SYNC))
    for name, eng in engines + engines[:2]:
        d = les.Domain(sc)
        if a.tile is not None:
            d.set_sor_config(a.tile, a.kc)
        net = les.Net(seed=0, stride=int(z["stride"]))
        net.set_params(z["params"])
        net.engine = eng
        for _ in range(a.warmup):
            d.step(1)
        d.set_warmstart(net)
        d.set_net_schedule(a.net_every)
        d.set_record(True)
        d.step(1)
        r = d.aux(les.LES_AUX_NET_IN)
        m = d.aux(les.LES_AUX_MASK)
        d.set_record(False)
        sw = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            sw.append(d.step(1)["sweeps"])
        torch.cuda.synchronize()
        ms_step = (time.perf_counter() - t0) * 1e3 / a.steps
        dr = torch.from_numpy(np.ascontiguousarray(r, np.float32)).cuda()
        dm = torch.from_numpy(np.ascontiguousarray(m, np.float32)).cuda()
        y = torch.empty_like(dr)
        for _ in range(3):
            les.les_net_forward(net.h, dr.data_ptr(), dm.data_ptr(), y.data_ptr(), sc.nx, sc.ny, sc.nz)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(20):
            les.les_net_forward(net.h, dr.data_ptr(), dm.data_ptr(), y.data_ptr(), sc.nx, sc.ny, sc.nz)
        ev1.record()
        torch.cuda.synchronize()
        out["rows"].append({"engine": name, "ms_per_step": ms_step, "sweeps": sw,
                            "forward_ms": ev0.elapsed_time(ev1) / 20, "y_norm": float(y.norm().item())})
        d.close()
        net.close()
    print(json.dumps(out))


def make(workload: str, seed: int):
    if workload == "lattice":
        return scene.lattice_scene(seed)
    if workload == "random":
        return scene.random_scene(seed)
    if workload == "large":
        return scene.large_scene(seed)
    if workload == "medium":
        # 384x384x128, periodic y: the SOR state (~170 MB of d, r and flags)
        # exceeds L2 while the whole handle stays near 2 GB (profiler captures)
        return scene.random_scene(seed=seed, nx=384, ny=384, nz=128, n_buildings=675, periodic_y=True)
    raise ValueError(workload)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="random", choices=["lattice", "random", "medium", "large", "ensemble"])
    ap.add_argument("--members", type=int, default=32, help="ensemble members")
    ap.add_argument("--max-sweeps", type=int, default=60000, help="ensemble members' sweep budget")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--graph", type=int, default=1)
    ap.add_argument("--tile", type=int, default=None)
    ap.add_argument("--kc", type=int, default=0)
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--range", action="store_true")
    ap.add_argument("--sweep-table", action="store_true",
                    help="time every SOR sweep configuration on the workload after the warm-up steps")
    ap.add_argument("--net", default=None, help="trained warm-start network (.npz: params, stride)")
    ap.add_argument("--net-every", type=int, default=0, help="network correction every n sweeps")
    ap.add_argument("--net-kernels", type=int, default=0,
                    help="les_set_net_kernels layout (0 folded, 1 persistent, 2 layers; + 4: the network's own pooling)")
    ap.add_argument("--sor-compare", default=None,
                    help="comma-separated sweep counts: red-black SOR vs the twinned double buffer "
                         "(les_sor_compare) from the previous step's pressure and the next step's rhs")
    ap.add_argument("--twin-omega", type=float, default=0.9, help="relaxation of the twinned double buffer")
    ap.add_argument("--fixed-sweeps", type=int, default=0,
                    help="run exactly this many SOR sweeps per step (0: solve to the tolerance)")
    ap.add_argument("--ens-tile", type=int, default=None, help="ensemble sweep mode (les_ensemble_set_tile)")
    ap.add_argument("--persistent", action="store_true", help="ensemble: plain steps as one persistent launch")
    ap.add_argument("--engines", action="store_true",
                    help="with --net: learned step time and network forward time for each convolution engine")
    a = ap.parse_args()
    if a.workload == "ensemble":
        return run_ensemble(a)
    if a.engines:
        return run_engines(a)
    sc = make(a.workload, a.seed)
    if a.fixed_sweeps > 0:
        sc.fixed_sweeps, sc.max_sweeps = 1, a.fixed_sweeps
    d = les.Domain(sc, precision=les.LES_FP64 if a.fp64 else les.LES_FP32, stream=None)
    d.set_graph(bool(a.graph))
    if a.tile is not None:
        d.set_sor_config(a.tile, a.kc)
    net = None
    if a.net:
        z = np.load(a.net)
        net = les.Net(seed=0, stream=None, stride=int(z["stride"]))
        net.set_params(z["params"])
    for _ in range(a.warmup):
        d.step(1)
    tune = None
    if a.sor_compare:
        # the pressure problem of a real step: the previous step's pressure and
        # the rhs (mean removed) the next step solves
        p_prev = d.fields()[3].astype(np.float64)
        d.step(1)
        rhs = d.aux(les.LES_AUX_RHS).astype(np.float64)
        rows = []
        for n in (int(x) for x in a.sor_compare.split(",")):
            for name, vid, om in (("red-black SOR", les.LES_SOR_REDBLACK, -1.0),
                                  ("twinned double buffer", les.LES_SOR_TWINNED, a.twin_omega)):
                _, ms, rel = d.sor_compare(vid, om, n, rhs, p_prev)
                rows.append({"variant": name, "omega": sc.omega if om <= 0 else om, "sweeps": n,
                             "ms_per_sweep": ms, "rel_residual": rel})
        _, ms17, rel17 = d.sor_compare(les.LES_SOR_TWINNED, 1.7, 20, rhs, p_prev)
        rows.append({"variant": "twinned double buffer", "omega": 1.7, "sweeps": 20, "ms_per_sweep": ms17,
                     "rel_residual": rel17})
        print(json.dumps({"workload": a.workload, "cells": sc.ncells, "sor_config": d.sor_config(), "rows": rows}))
        return
    if a.sweep_table:
        rows = []
        for t in range(-1, les.LES_SOR_NTILES):
            for kc in ((0, 8, 16) if (0 <= t <= 5 or 25 <= t < 29) else (0,)):
                try:
                    ms = d.time_sor(t, kc, sweeps=20)
                except les.LesError:
                    continue
                rows.append({"tile": t, "kc": kc, "shape": les.les_sor_tile(t) if t >= 0 else "two-pass",
                             "ms_per_sweep": ms, "alg_gbs": 13.0 * sc.ncells / (ms * 1e-3) / 1e9})
        print(json.dumps({"workload": a.workload, "cells": sc.ncells, "sweep_table": rows}))
        return
    if a.autotune:
        tune = d.autotune_sor(sweeps=20)
    if net is not None:
        d.set_warmstart(net)
        d.set_net_schedule(a.net_every)
        d.set_net_kernels(a.net_kernels)
        d.step(1)
    if a.range:
        les.les_profiler_range(1)
    t0 = time.perf_counter()
    sweeps = []
    for _ in range(a.steps):
        st = d.step(1)
        sweeps.append(st["sweeps"])
    t1 = time.perf_counter()
    if a.range:
        les.les_profiler_range(0)
    err = les.les_last_error(d.h)
    print(json.dumps({"workload": a.workload, "graph_used": st["graph"], "last_error": err, "cells": sc.ncells, "steps": a.steps,
                      "ms_per_step": (t1 - t0) * 1e3 / a.steps, "sweeps": sweeps,
                      "rel_residual": st["rel_residual"], "sor_config": d.sor_config(), "autotune": tune,
                      "graph": a.graph, "net": a.net, "net_every": a.net_every}))


if __name__ == "__main__":
    main()
