"""Throughput of the LES time step on GB300: Mcell-steps/s with every step's
SOR solved to relative residual 1e-6 (so |div u| <= 1e-6 relative after each
projection).

Workload: the paper's default domain size (150 x 150 x 90, Sec. 2.7) with 100
random cuboid buildings at 30% plan density, stretched dz 2->8 m, log-law
inflow with 10% turbulence; all inputs synthetic and seeded (scene.py).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  ``value`` times each step with CUDA events on
the library's stream, the fields resident in HBM, L2 flushed (256 MiB write)
before every timed step.  ``e2e`` times the same K steps through the C ABI
with pinned host buffers: les_set_fields (H2D) + les_step + les_get_fields
(D2H).  The CPU legs run the FP64 oracle (OpenMP build, every host core):
``cpu_baseline`` is one real oracle step of the same state to the same stop
test, and ``oracle_err`` compares the GPU's results with the oracle's.
``--impl reference`` times real oracle steps of the workload on every host
core (see run_reference).
"""

from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1504_02264_gb300 import scene  # noqa: E402

METRIC = "LES Mcell-steps/s to |div|<=1e-6 (150x150x90, 100 buildings)"
WEIGHTS = os.path.join(ROOT, "paper_1504_02264_gb300", "weights", "warmstart.npz")
NET_EVERY = 10                  # sweeps between learned corrections (trained schedule)
UNIT = "Mcell-steps/s"
SOR_BYTES_PER_CELL = 13.0       # per sweep: read p, rhs (4+4), flags (1), write p (4)
# DRAM bytes (read + write) per launch of the TMA sweep kernels on this
# workload, by tile, from one ncu capture each (cold L2); reported only for the
# tile the autotuner picked
SOR_DRAM_BYTES = {17: 20.180736e6 + 3.072e3, 29: 20.188160e6, 30: 20.184832e6, 31: 20.187904e6, 32: 20.184320e6,
                  33: 20.184832e6, 34: 20.185088e6}
# the sweep timed alone on the HBM-bound grid: the column-walk TMA block
SOR_HBM_TILE = 29
L2_FLUSH_BYTES = 256 << 20
# algorithmic bytes per cell of the HBM-bound phases (every array read or
# written once): the stencil phase = les (u, v, w, flags in; nu_t out: 17 B)
# + velfg/SGS/Adams-Bashforth/feedbf (u, v, w, nu_t, flags, F^{n-1} in; F^n,
# u* out: 53 B) + rhs (u*, flags in; rhs out: 17 B); the projection (u*, p,
# flags in; u and the gauged p out: 41 B)
STENCIL_BYTES_PER_CELL = 17.0 + 53.0 + 17.0
PROJECT_BYTES_PER_CELL = 41.0


def workload(seed=0):
    sc = scene.random_scene(seed=seed)          # 150 x 150 x 90, tol 1e-6
    sc.check_every = 10
    sc.max_sweeps = 20000
    return sc


def small_workload(seed=0):
    """A 48x48x24 random city with the same recipe (host-logic tests only)."""
    sc = scene.random_scene(seed=seed, nx=48, ny=48, nz=24, n_buildings=8, x_margin=8)
    sc.check_every = 10
    sc.max_sweeps = 20000
    return sc


def sor_kernel_name(tile):
    """The sweep kernel a tile index of les_set_sor_config runs."""
    if tile >= 29:
        return "k_sor_col"
    if tile >= 25:
        return "k_sor_march"
    if tile >= 21:
        return "k_sor_pipe"
    if tile >= 17:
        return "k_sor_tma"
    if tile >= 12:
        return "k_sor_rows"
    if tile >= 6:
        return "k_sor_block"
    return "k_sor_fused" if tile >= 0 else "k_sor_half"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_cpu():
    """Host cores and CPU model (lscpu when present, else /proc/cpuinfo)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"nproc": cores, "model": model or "unknown", "machine": platform.machine()}


# ---------------------------------------------------------------------------
# nvidia-smi clock sampling during the timed region

class Clocks:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, interval_ms=50):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", str(interval_ms)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU legs: the FP64 oracle (OpenMP build on every host core)

def oracle_threads():
    from oracle import oracle as orc
    n = host_cpu()["nproc"]
    orc.set_threads(n)
    return orc.threads(True)


def oracle_from_state(sc, state):
    """An OpenMP oracle domain holding a GPU state (fields, AB2 history, step)."""
    from oracle.oracle import Oracle, A_FU, A_FV, A_FW
    o = Oracle(sc, omp=True)
    o.set_fields(*state["fields"])
    for a, arr in zip((A_FU, A_FV, A_FW), state["F"]):
        o.set(a, arr)
    o.step_index = state["step"]
    return o


def oracle_step_timed(o):
    """One real oracle step to the stop test, timed phase by phase."""
    t0 = time.perf_counter()
    o.bc_fill()
    o.les_nut()
    o.momentum()
    o.outflow_fix()
    o.make_rhs()
    t1 = time.perf_counter()
    o.sor_solve()
    t2 = time.perf_counter()
    o.project()
    o.step_index = o.step_index + 1
    t3 = time.perf_counter()
    st = o.stats()
    return t3 - t0, {"prefix_s": t1 - t0, "sor_s": t2 - t1, "project_s": t3 - t2, "sweeps": st["sweeps"],
                     "rel_residual": st["rel_residual"]}


def field_errors(gpu_fields, ref_fields):
    """Max relative velocity error (over u, v, w, scaled by the largest
    velocity) and max relative error of the gauged pressure."""
    g = [np.asarray(a, np.float64) for a in gpu_fields]
    vel = max(np.abs(a).max() for a in ref_fields[:3])
    ev = max(np.abs(a - b).max() for a, b in zip(g[:3], ref_fields[:3])) / vel
    ep = np.abs(g[3] - ref_fields[3]).max() / max(np.abs(ref_fields[3]).max(), 1e-300)
    return float(ev), float(ep)


def oracle_divergence(sc, fields):
    """FP64 oracle's |div u| (2-norm over cells) of a velocity field, and the
    part of it FP32 storage of the face values alone can leave: the 2-norm of
    2^-24 times the sum of |face value| / spacing over each fluid cell."""
    from oracle.oracle import Oracle
    o = Oracle(sc, omp=True)
    u, v, w, p = [np.asarray(a, np.float64) for a in fields]
    o.set_fields(u, v, w, p)
    dz = np.asarray(sc.dz, np.float64)[:, None, None]
    mag = ((np.abs(u[:, :, 1:]) + np.abs(u[:, :, :-1])) / sc.dx + (np.abs(v[:, 1:]) + np.abs(v[:, :-1])) / sc.dy +
           (np.abs(w[1:]) + np.abs(w[:-1])) / dz) * (sc.solid == 0)
    return float(np.linalg.norm(o.divergence())), float(2.0 ** -24 * np.linalg.norm(mag))


def lattice_parity(les):
    """Config 1 (64x64x32 lattice, 20 steps x 50 sweeps, FP32 with the sweep
    kernel the autotuner picks) against the FP64 oracle."""
    from oracle.oracle import Oracle
    sc = scene.lattice_scene(0)
    o = Oracle(sc, omp=True)
    o.step(20)
    d = les.Domain(sc)
    try:
        (tile, kc), _ = d.autotune_sor(sweeps=20)
        d.step(20)
        g = d.fields()
    finally:
        d.close()
    ev, ep = field_errors(g, o.fields())
    return {"workload": "lattice_64x64x32 (20 steps, 50 sweeps each)", "sor_tile": tile,
            "max_rel_velocity_err": ev, "max_rel_pressure_err": ep, "bar": 1e-4}


# ---------------------------------------------------------------------------
# the HBM-bound grid (config 3: 512 x 512 x 128, periodic y)

def hbm_large(les, net, peak, peak_kind, steps):
    """The HBM-bound kernels where the state does not fit in L2, and the
    converged step rate.  (1) 20 fixed sweeps per step, host loop with CUDA
    events around each phase (stencil phase: bondv1, les, velfg/SGS/AB2/
    feedbf, outflow, rhs; projection), and the SOR sweep of the column-walk TMA block
    tile timed alone (20 back-to-back sweeps, best of 3).  (2) Steps to
    relative residual 1e-6, learned and plain, from the same state."""
    import torch
    sc = scene.large_scene(0)
    sc.fixed_sweeps, sc.max_sweeps = 1, 20
    d = les.Domain(sc)
    try:
        d.set_graph(False)
        d.step(1)
        d.set_timing(True)
        d.step(2)
        tm = d.timing()
        d.set_timing(False)
        sweep_ms = min(d.time_sor(SOR_HBM_TILE, 0, sweeps=20) for _ in range(3))
    finally:
        d.close()
    n = sc.ncells
    nsteps = max(tm["steps"], 1)

    def entry(bytes_per_cell, ms):
        gbs = bytes_per_cell * n / (ms * 1e-3) / 1e9
        return {"ms": ms, "bytes_per_cell": bytes_per_cell, "achieved_gbs": gbs, "frac": gbs / peak}

    out = {"workload": "large_512x512x128_periodic_y", "cells": n, "peak_gbs": peak, "peak_kind": peak_kind,
           "l2": "state (~3.5 GB) far larger than L2",
           "sor_sweep": {"kernel": f"{sor_kernel_name(SOR_HBM_TILE)} tile {les.les_sor_tile(SOR_HBM_TILE)}",
                         **entry(SOR_BYTES_PER_CELL, sweep_ms)},
           "stencil_phase": entry(STENCIL_BYTES_PER_CELL, tm["ms_momentum"] / nsteps),
           "projection": {**entry(PROJECT_BYTES_PER_CELL, tm["ms_project"] / nsteps),
                          "note": "FP64 pressure differences: bound by the FP64 pipe, not HBM"}}

    # converged steps (tolerance 1e-6 every step)
    sc = scene.large_scene(0)
    sc.check_every, sc.max_sweeps = 10, 400000
    d = les.Domain(sc)
    try:
        d.step(1)
        d.autotune_sor(sweeps=10)
        state = d.get_state()
        conv = {}
        for mode, k in (("learned", steps), ("plain", 1)):
            d.set_state(state)
            if mode == "learned":
                d.set_warmstart(net)
                d.set_net_schedule(NET_EVERY)
                d.step(1)                      # builds its graphs
                d.set_state(state)
            else:
                d.set_warmstart(None)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
            sw, worst = [], 0.0
            stream = torch.cuda.current_stream()
            for s in range(k):
                ev[s][0].record(stream)
                st = d.step(1)
                ev[s][1].record(stream)
                if st["rc"] != 0:
                    raise RuntimeError(f"large {mode} step did not converge: {st}")
                sw.append(st["sweeps"])
                worst = max(worst, st["rel_residual"])
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev) / k
            conv[mode] = {"steps": k, "ms_per_step": ms, "mcell_steps_per_s": n / (ms * 1e-3) / 1e6,
                          "mean_sweeps_per_step": float(np.mean(sw)), "max_rel_residual": worst}
        conv["learned_speedup_vs_plain"] = conv["plain"]["ms_per_step"] / conv["learned"]["ms_per_step"]
        conv["note"] = ("tolerance 1e-6 every step, from the state after one plain step; CUDA graphs; "
                        "plain: previous-step pressure start")
        out["converged"] = conv
    finally:
        d.close()
    return out


# ---------------------------------------------------------------------------
# config 4: the batched ensemble of uneven domains

def ensemble_leg(les, net, steps):
    """32 uneven random cities (96^2-256^2 x 64-128, own buildings and inflow)
    stepped together, learned correction and plain SOR from the same state."""
    import torch
    scs = scene.ensemble_scenes(seed=0, n=32)
    for sc in scs:
        sc.max_sweeps = 60000
    cells = sum(sc.ncells for sc in scs)
    ens = les.Ensemble(scs)
    try:
        ens.set_warmstart(net, NET_EVERY)
        ens.step(1)
        tune = ens.autotune(sweeps=10)
        states = [m.get_state() for m in ens.members]
        out = {"workload": "ensemble_32_uneven", "members": len(scs), "cells": cells,
               "shapes_min_max": [min(sc.ncells for sc in scs), max(sc.ncells for sc in scs)],
               "tile": tune[0], "autotune_ms_per_sweep": tune[1]}
        for mode, k in (("learned", steps), ("plain", 1)):
            for m, s in zip(ens.members, states):
                m.set_state(s)
            if mode == "plain":
                ens.set_warmstart(None)
            l0 = ens.launches()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sw, worst = [], 0.0
            for _ in range(k):
                st = ens.step(1)
                if st[0]["rc"] != 0:
                    raise RuntimeError(f"ensemble {mode} step did not converge")
                sw.append(max(x["sweeps"] for x in st))
                worst = max(worst, max(x["rel_residual"] for x in st))
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / k
            out[mode] = {"steps": k, "ms_per_step": ms, "mcell_steps_per_s": cells / (ms * 1e-3) / 1e6,
                         "slowest_member_sweeps": float(np.mean(sw)), "max_rel_residual": worst,
                         "launches_per_step": (ens.launches() - l0) / k}
        # the plain step again as one persistent cooperative launch per step
        for m, s in zip(ens.members, states):
            m.set_state(s)
        ens.set_persistent(True)
        l0 = ens.launches()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ens.step(1)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        if st[0]["rc"] != 0:
            raise RuntimeError("ensemble persistent step did not converge")
        out["plain_persistent"] = {"steps": 1, "ms_per_step": ms, "mcell_steps_per_s": cells / (ms * 1e-3) / 1e6,
                                   "slowest_member_sweeps": float(max(x["sweeps"] for x in st)),
                                   "max_rel_residual": max(x["rel_residual"] for x in st),
                                   "launches_per_step": ens.launches() - l0,
                                   "note": "the whole SOR solve of all members in one cooperative launch"}
        ens.set_persistent(False)
        out["learned_speedup_vs_plain"] = out["plain"]["ms_per_step"] / out["learned"]["ms_per_step"]
        out["note"] = "host wall time around ens.step (CUDA graphs inside); tolerance 1e-6 per member"
    finally:
        ens.close()
    return out


# ---------------------------------------------------------------------------
# multi-rank helpers (replicas: one independent domain per rank, weak scaling)

def replica_seed(rank):
    """Scene seed of a rank's replica: the ranks step different cities."""
    return rank


def max_over_ranks(x, dist, device):
    """The slowest rank's time (every rank gets it)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mcell_steps(cells_per_rank, world, ms_per_step):
    """Whole-job throughput: the cells of all ranks per step over the slowest
    rank's step time."""
    return cells_per_rank * world / (ms_per_step * 1e-3) / 1e6


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle, real steps

def run_reference(args):
    """Real oracle steps of the workload (OpenMP build, every host core): each
    timed step runs bondv1 ... press to the same stop test (relative residual
    1e-6, checked every 10 sweeps) and velnw, from the workload's initial
    state.  A full step takes minutes on the CPU, so the run times at most K
    steps and stops early once ``--ref-budget-s`` seconds are spent (at least
    one step); ``steps`` reports the steps timed.  The W warm-up steps are
    one-sweep steps of a separate oracle domain (thread pool and caches)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle.oracle import Oracle
    sc = small_workload() if args.ref_workload == "small" else workload()
    n = sc.ncells
    cores = oracle_threads()
    cpu = host_cpu()
    warm = Oracle(sc, omp=True, fixed_sweeps=1, max_sweeps=1)
    for _ in range(args.warmup):
        warm.step(1)
    del warm
    o = Oracle(sc, omp=True)
    times, sweeps, t_all = [], [], time.perf_counter()
    for s in range(args.steps):
        t, det = oracle_step_timed(o)
        times.append(t)
        sweeps.append(det["sweeps"])
        if time.perf_counter() - t_all > args.ref_budget_s:
            break
    t = float(np.mean(times))
    val = n / t / 1e6
    name = "random_150x150x90" if args.ref_workload != "small" else "random_48x48x24"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded scene.py)",
            "config": {"workload": name, "nx": sc.nx, "ny": sc.ny, "nz": sc.nz, "tol": sc.tol,
                       "check_every": sc.check_every, "l2": "n/a (CPU)"},
            "sweeps_per_step": sweeps,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "nproc": cpu["nproc"], "cpu_model": cpu["model"], "machine": cpu["machine"],
                             "sample": (f"{len(times)} real FP64 oracle step(s) of the workload from its initial "
                                        f"state, each solved to relative residual {sc.tol:g} (OpenMP build, "
                                        f"{cores} threads); budget {args.ref_budget_s:g} s")},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1504_02264_gb300 import les

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    # independent domain per rank (weak scaling: replicas, no data-path collective)
    sc = workload(seed=replica_seed(rank))
    n = sc.ncells
    dom = les.Domain(sc, precision=les.LES_FP32)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        st = dom.step(1)
        if st["rc"] < 0:
            raise RuntimeError(st)
    # set-up, not timed: pick the SOR tile shape and k-chunk for this grid
    (tile, kc), tune_ms = dom.autotune_sor(sweeps=20)
    net = None
    if not args.no_learned:
        from paper_1504_02264_gb300 import train
        net = train.load(WEIGHTS)
    state0 = dom.get_state()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    def timed(label, clocks_on, k):
        """k steps from state0, each bracketed by CUDA events on the library's
        stream after an L2 flush; max over ranks."""
        dom.set_state(state0)
        l0 = dom.timing()["launches"]
        clocks = Clocks(local) if (clocks_on and rank == 0 and not args.ncu_range) else None
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        sweeps, worst, graph_used = [], 0.0, 0
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        if args.ncu_range:
            torch.cuda.profiler.start()
        for s in range(k):
            flush.zero_()
            ev[s][0].record(stream)
            st = dom.step(1)
            ev[s][1].record(stream)
            sweeps.append(st["sweeps"])
            graph_used = st["graph"]
            worst = max(worst, st["rel_residual"])
            if st["rc"] != 0:
                raise RuntimeError(f"{label} step did not converge: {st}")
        torch.cuda.synchronize()
        if args.ncu_range:
            torch.cuda.profiler.stop()
        clk = clocks.stop() if clocks else None
        launches = dom.timing()["launches"] - l0
        ms = sum(a.elapsed_time(b) for a, b in ev) / k
        if world > 1:
            ms = max_over_ranks(ms, dist, dev)
        return {"ms": ms, "sweeps": sweeps, "worst": worst, "graph": graph_used, "clocks": clk,
                "launches": launches}

    def use_net(nw):
        dom.set_warmstart(nw)
        dom.set_net_schedule(NET_EVERY)
        dom.set_state(state0)
        dom.step(1)                    # builds its graphs (untimed)

    # timed region 1: the plain step (red-black SOR from the previous
    # pressure, one chunked CUDA graph per step)
    plain = timed("plain", True, args.steps)
    ablation = None
    if net is not None:
        # timed region 1b: the full hot path with the learned correction
        # (the package's network every NET_EVERY sweeps), same start state, same
        # stop test
        use_net(net)
        learned = timed("learned", True, args.steps)
        head = learned
        # the same, with each prediction overlapped with the next batch of sweeps
        dom.set_net_async(True)
        use_net(net)
        overlapped = timed("learned_overlapped", True, args.steps)
        dom.set_net_async(False)
        if overlapped["ms"] < learned["ms"]:
            head = overlapped
        # what the training buys: the same correction cycle with untrained
        # (He-normal) weights and with the non-learned coarse correction
        # q = prolongated pooled residual
        if not args.no_ablation:
            from paper_1504_02264_gb300 import train
            ablation = {}
            k_abl = max(1, min(args.steps, 5))
            for name in ("untrained", "coarse_residual"):
                other = les.Net(seed=123, stride=net.stride)
                if name == "coarse_residual":
                    other.set_params(train.coarse_residual_params(other.nparam))
                use_net(other)
                r = timed(name, False, k_abl)
                ablation[name] = {"ms_per_step": r["ms"], "mean_sweeps_per_step": float(np.mean(r["sweeps"])),
                                  "steps": k_abl}
                dom.set_warmstart(None)
                torch.cuda.synchronize()
                other.close()
            ablation["trained"] = {"ms_per_step": learned["ms"],
                                   "mean_sweeps_per_step": float(np.mean(learned["sweeps"])), "steps": args.steps}
            ablation["note"] = ("same cycle (every 10 sweeps, stride 8, energy-norm step, same kernels); "
                                "untrained = He-normal weights (seed 123); coarse_residual = weights that make "
                                "the network return the pooled residual / rms")
            use_net(net)
    else:
        head = plain
    head_async = net is not None and head is overlapped
    ms, sweeps, worst, graph_used, clk, launches = (head["ms"], head["sweeps"], head["worst"], head["graph"],
                                                    head["clocks"], head["launches"])
    net_phases = None
    if net is not None:
        # phase times of the learned step (host loop with CUDA events around
        # each phase; not the timed region)
        dom.set_state(state0)
        dom.set_timing(True)
        for s in range(min(args.steps, 3)):
            flush.zero_()
            dom.step(1)
        torch.cuda.synchronize()
        tn = dom.timing()
        dom.set_timing(False)
        net_phases = {k: tn[k] / max(tn["steps"], 1) for k in
                      ("ms_momentum", "ms_sor", "ms_residual", "ms_project", "ms_net")}
        net_phases["net_cycles_per_step"] = tn["net_cycles"] / max(tn["steps"], 1)
        net_phases["sweeps_per_step"] = tn["sor_sweeps"] / max(tn["steps"], 1)
        net_phases["note"] = "host loop with an event pair around every phase; sums exceed the graph step time"
        # the SOR kernel roofline uses the plain step
        dom.set_warmstart(None)
        dom.set_state(state0)

    # timed region 2: same steps, host-driven, with CUDA events around every
    # batch of SOR sweep launches on the library's stream (kernel roofline:
    # the plain step's sweeps, the same kernel and tile the graphs launch)
    dom.set_timing(True)
    for s in range(min(args.steps, 3)):
        flush.zero_()
        dom.step(1)
    torch.cuda.synchronize()
    tm = dom.timing()
    dom.set_timing(False)

    # the GPU's own result of one step from state0, plain and learned (for the
    # oracle comparison of the CPU legs)
    step_out = {}
    if not args.no_cpu_baseline and rank == 0:
        for mode in ("plain",) + (("learned",) if net is not None else ()):
            dom.set_warmstart(net if mode == "learned" else None)
            if mode == "learned":
                dom.set_net_schedule(NET_EVERY)
                dom.set_net_async(head_async)
            dom.set_state(state0)
            st = dom.step(1)
            step_out[mode] = {"fields": dom.fields(), "stats": st,
                              "ustar": [dom.aux(a) for a in (les.LES_AUX_USTAR, les.LES_AUX_VSTAR,
                                                             les.LES_AUX_WSTAR)]}
        dom.set_warmstart(None)

    # end to end through the C ABI with pinned host buffers (the configuration
    # of the headline value), the same K steps
    if net is not None:
        dom.set_warmstart(net)
        dom.set_net_schedule(NET_EVERY)
        dom.set_net_async(head_async)
    dom.set_state(state0)
    dom.step(1)                        # builds the configuration's graphs (untimed)
    dom.set_state(state0)
    shapes = dom.shapes()
    host = [torch.empty(s, dtype=torch.float32, pin_memory=True).numpy() for s in shapes]
    for h, f in zip(host, dom.fields()):
        h[...] = f
    h2d = sum(h.nbytes for h in host)
    torch.cuda.synchronize()
    ee = []
    for s in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        les.les_set_fields(dom.h, *host)
        les.les_step(dom.h, 1, les.les_stats_t())
        les.les_get_fields(dom.h, *host)
        b.record(stream)
        b.synchronize()
        ee.append(a.elapsed_time(b))
    e2e_ms = float(np.mean(ee))
    if world > 1:
        e2e_ms = max_over_ranks(e2e_ms, dist, dev)

    if rank == 0:
        peak, peak_kind = peaks()
        sweep_ms = tm["ms_sor"] / max(tm["sor_sweeps"], 1)
        launch_ms = tm["ms_sor"] / max(tm["sor_launches"], 1)
        launches_per_sweep = tm["sor_launches"] / max(tm["sor_sweeps"], 1)
        bytes_per_launch = SOR_BYTES_PER_CELL * n / launches_per_sweep
        achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9
        mean_sweeps = float(np.mean(sweeps))
        plain_sweeps = float(np.mean(plain["sweeps"]))
        line = {
            "metric": METRIC, "value": aggregate_mcell_steps(n, world, ms), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 norms)",
            "data": "synthetic (seeded scene.py: random city, log-law inflow, 10% turbulence)",
            "config": {"workload": "random_150x150x90", "nx": 150, "ny": 150, "nz": 90, "buildings": 100,
                       "tol": 1e-6, "check_every": sc.check_every, "mean_sweeps_per_step": mean_sweeps,
                       "max_rel_residual": worst, "parallelism": f"replicas x{world}",
                       "sor_start": (f"previous-step pressure + learned correction (U-Net at stride {net.stride} "
                                     f"every {NET_EVERY} sweeps"
                                     f"{', each prediction overlapped with the next sweeps' if head_async else ''})"
                                     if net is not None else "previous-step pressure"),
                       "l2": "flushed (256 MiB write) before every timed step"},
            "plain_sor": {"value": aggregate_mcell_steps(n, world, plain["ms"]), "unit": UNIT,
                          "ms_per_step": plain["ms"], "mean_sweeps_per_step": plain_sweeps,
                          "max_rel_residual": plain["worst"],
                          "step_mode": "cuda_graph" if plain["graph"] else "host_loop",
                          "gpu_launches": int(plain["launches"]), "clocks": plain["clocks"]},
            "learned": None if net is None else {
                "ms_per_step": ms, "mean_sweeps_per_step": mean_sweeps,
                "schedule": "overlapped" if head is overlapped else "in_place",
                "in_place": {"ms_per_step": learned["ms"], "mean_sweeps_per_step": float(np.mean(learned["sweeps"]))},
                "overlapped": {"ms_per_step": overlapped["ms"],
                               "mean_sweeps_per_step": float(np.mean(overlapped["sweeps"])),
                               "note": "each network prediction runs on a second stream during the next batch "
                                       "of sweeps and is applied after it (les_set_net_async)"},
                "speedup_vs_plain_sor": plain["ms"] / ms, "sweeps_ratio": plain_sweeps / max(mean_sweeps, 1.0),
                "net_every_sweeps": NET_EVERY, "stride": net.stride,
                "weights": os.path.relpath(WEIGHTS, ROOT),
                "note": "same start state and stop test (FP64 relative residual <= 1e-6 every step); "
                        "network time included",
                "ablation": ablation,
                "phase_ms_per_step": net_phases},
            "roofline": {"kernel": f"{sor_kernel_name(tile)} (red-black SOR sweep, tile "
                                   f"{les.les_sor_tile(tile) if tile >= 0 else 'two-pass'}, kc {kc})",
                         "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind,
                         "traffic": SOR_DRAM_BYTES.get(tile),
                         "bytes_per_launch": bytes_per_launch, "launch_ms": launch_ms,
                         "note": ("150x150x90 SOR state (p, rhs, flags ~18 MB) is L2-resident; timed on the "
                                  "plain step's sweep batches (host loop, events around each batch)")},
            "phase_ms_per_step": {k: tm[k] / max(tm["steps"], 1) for k in
                                  ("ms_momentum", "ms_sor", "ms_residual", "ms_project")},
            "sor_ms_per_sweep": sweep_ms,
            "gpu_launches": int(launches),
            "step_mode": "cuda_graph" if graph_used else "host_loop",
            "sor_autotune": {"tile": tile, "kc": kc, "ms_per_sweep": tune_ms},
            "e2e": {"value": aggregate_mcell_steps(n, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": h2d, "ms_per_step": e2e_ms, "steps": args.steps},
            "clocks": clk,
        }
        if not args.no_cpu_baseline:
            line.update(cpu_legs(les, sc, dom, state0, step_out))
        if not args.no_large:
            line["hbm_large"] = hbm_large(les, net, peak, peak_kind, steps=3)
        if not args.no_ensemble and net is not None:
            line["ensemble"] = ensemble_leg(les, net, steps=2)
        print(json.dumps(line))
    dom.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def cpu_legs(les, sc, dom, state0, step_out):
    """One real oracle step from the GPU's post-warm-up state (the CPU
    baseline) and the errors of the GPU's results against the oracle."""
    from oracle.oracle import A_US, A_VS, A_WS
    cores = oracle_threads()
    cpu = host_cpu()
    dom.set_state(state0)
    state = {"fields": [f.astype(np.float64) for f in dom.fields()],
             "F": [dom.aux(a).astype(np.float64) for a in (les.LES_AUX_FU, les.LES_AUX_FV, les.LES_AUX_FW)],
             "step": dom.step(0)["step"]}
    o = oracle_from_state(sc, state)
    t_step, det = oracle_step_timed(o)
    ref = o.fields()
    ref_star = [o.get(a) for a in (A_US, A_VS, A_WS)]      # u*, v*, w* of the oracle's step
    out = {"cpu_baseline": {
        "value": sc.ncells / t_step / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
        "nproc": cpu["nproc"], "cpu_model": cpu["model"], "machine": cpu["machine"],
        "sample": (f"one real FP64 oracle step (OpenMP build, {cores} threads) of the same 150x150x90 state the "
                   f"timed GPU steps start from, solved to relative residual {sc.tol:g}: "
                   f"{det['sweeps']} sweeps, {t_step:.1f} s"),
        "detail": det}}
    err = {"reference": f"the oracle's step from the same state (FP64, same stop test: {det['sweeps']} sweeps)",
           "note": ("max relative errors of the GPU step's fields against the oracle's; rel_div_by_oracle = "
                    "|div u^{n+1}| / |div u*| with both divergences formed by the oracle from the GPU's FP32 "
                    "fields, next to the share of it that FP32 rounding of the face values alone can leave")}
    vel = max(np.abs(a).max() for a in state["fields"][:3])
    for mode, r in step_out.items():
        ev, ep = field_errors(r["fields"], ref)
        es = max(float(np.abs(a.astype(np.float64) - b).max()) for a, b in zip(r["ustar"], ref_star)) / vel
        div_star, _ = oracle_divergence(sc, [a.astype(np.float64) for a in r["ustar"]] + [ref[3]])
        div, floor = oracle_divergence(sc, r["fields"])
        err[mode] = {"max_rel_velocity_err": ev, "max_rel_pressure_err": ep, "ustar_max_rel_err": es,
                     "rel_div_by_oracle": div / max(div_star, 1e-300),
                     "rel_div_fp32_floor": floor / max(div_star, 1e-300), "sweeps": r["stats"]["sweeps"]}
    err["lattice_config1"] = lattice_parity(les)
    out["oracle_err"] = err
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle legs")
    ap.add_argument("--no-learned", action="store_true", help="time the plain SOR step only")
    ap.add_argument("--no-ablation", action="store_true", help="skip the untrained / non-learned cycles")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 512x512x128 grid (HBM-bound kernels, converged steps)")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 32-member ensemble")
    ap.add_argument("--ref-budget-s", type=float, default=240.0,
                    help="reference arm: stop timing oracle steps after this many seconds")
    ap.add_argument("--ref-workload", default="bench", choices=["bench", "small"],
                    help="reference arm workload (small: a 48x48x24 city, host-logic tests)")
    ap.add_argument("--ncu-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
