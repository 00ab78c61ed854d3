"""Throughput of the LES time step on GB300: Mcell-steps/s with every step's
SOR solved to relative residual 1e-6 (so |div u| <= 1e-6 relative after each
projection).

Workload: the paper's default domain size (150 x 150 x 90, Sec. 2.7) with 100
random cuboid buildings at 30% plan density, stretched dz 2->8 m, log-law
inflow with 10% turbulence; all inputs synthetic and seeded (scene.py).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  ``value`` times each step with CUDA events on
the library's stream, the fields resident in HBM, L2 flushed (256 MiB write)
before every timed step.  ``e2e`` times the same steps through the C ABI with
pinned host buffers: les_set_fields (H2D) + les_step + les_get_fields (D2H).
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (see ``cpu_sample``).
"""

from __future__ import annotations

import argparse
import json
import os
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
# DRAM bytes (read + write) of one k_sor_tma launch on this workload from one
# ncu capture (cold L2; profiles/sor_tma_28x8x8_random150x150x90.md); reported
# only while that kernel is the one timed
SOR_TMA_TILE, SOR_TMA_DRAM_BYTES = 17, 20.180480e6 + 1.536e3
L2_FLUSH_BYTES = 256 << 20
# algorithmic bytes per cell of the HBM-bound phases (every array read or
# written once): the stencil phase = les (u, v, w, flags in; nu_t out: 17 B)
# + velfg/SGS/Adams-Bashforth/feedbf (u, v, w, nu_t, flags, F^{n-1} in; F^n,
# u* out: 53 B) + rhs (u*, flags in; rhs out: 17 B); the projection (u*, p,
# flags in; u and the gauged p out: 41 B)
STENCIL_BYTES_PER_CELL = 17.0 + 53.0 + 17.0
PROJECT_BYTES_PER_CELL = 41.0
# mean SOR sweeps per step of this workload after the default warm-up, from the
# GPU arm (the FP64 path takes the same sweeps as the oracle); used only to scale
# the bounded oracle sample to a full step when no GPU run is available
REF_SWEEPS_PER_STEP = 12600


def workload(seed=0):
    sc = scene.random_scene(seed=seed)          # 150 x 150 x 90, tol 1e-6
    sc.check_every = 10
    sc.max_sweeps = 20000
    return sc


def sor_kernel_name(tile):
    """The sweep kernel a tile index of les_set_sor_config runs."""
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
# CPU oracle, bounded sample

def oracle_sample(sc, sweeps_per_step, n_sample_sweeps=40, state=None):
    """Time one oracle step phase by phase with a fixed SOR sample and scale the
    SOR part to ``sweeps_per_step``.  Returns (seconds per full step, detail)."""
    from oracle.oracle import Oracle, A_FU, A_FV, A_FW

    o = Oracle(sc, fixed_sweeps=1, max_sweeps=n_sample_sweeps)
    if state is not None:
        o.set_fields(*state["fields"])
        for a, arr in zip((A_FU, A_FV, A_FW), state["F"]):
            o.set(a, arr)
        o.step_index = state["step"]
    t0 = time.perf_counter()
    o.bc_fill()
    o.les_nut()
    o.momentum()
    o.outflow_fix()
    o.make_rhs()
    t1 = time.perf_counter()
    o.sor_sweeps(n_sample_sweeps)
    t2 = time.perf_counter()
    o.residual()
    t3 = time.perf_counter()
    o.gauge()
    o.project()
    t4 = time.perf_counter()
    t_sweep = (t2 - t1) / n_sample_sweeps
    checks = sweeps_per_step / max(sc.check_every, 1)
    t_step = (t1 - t0) + (t4 - t3) + sweeps_per_step * t_sweep + checks * (t3 - t2)
    return t_step, {"non_sor_s": (t1 - t0) + (t4 - t3), "sweep_s": t_sweep, "residual_s": t3 - t2,
                    "sample_wall_s": t4 - t0}


def hbm_large(peak, peak_kind):
    """The HBM-bound kernels where the state does not fit in L2: the
    512x512x128 periodic-y city (1200 buildings), 20 fixed sweeps per step,
    host loop with CUDA events around each phase (stencil phase: bondv1, les,
    velfg/SGS/AB2/feedbf, outflow, rhs; projection), and the SOR sweep of the
    TMA block tile timed alone (20 back-to-back sweeps, best of 3)."""
    from paper_1504_02264_gb300 import les
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
        sweep_ms = min(d.time_sor(SOR_TMA_TILE, 0, sweeps=20) for _ in range(3))
    finally:
        d.close()
    n = sc.ncells
    steps = max(tm["steps"], 1)

    def entry(bytes_per_cell, ms):
        gbs = bytes_per_cell * n / (ms * 1e-3) / 1e9
        return {"ms": ms, "bytes_per_cell": bytes_per_cell, "achieved_gbs": gbs, "frac": gbs / peak}

    return {"workload": "large_512x512x128_periodic_y", "cells": n, "peak_gbs": peak, "peak_kind": peak_kind,
            "l2": "state (~3.5 GB) far larger than L2",
            "sor_sweep": {"kernel": f"{sor_kernel_name(SOR_TMA_TILE)} tile {les.les_sor_tile(SOR_TMA_TILE)}",
                          **entry(SOR_BYTES_PER_CELL, sweep_ms)},
            "stencil_phase": entry(STENCIL_BYTES_PER_CELL, tm["ms_momentum"] / steps),
            "projection": {**entry(PROJECT_BYTES_PER_CELL, tm["ms_project"] / steps),
                           "note": "FP64 pressure differences: bound by the FP64 pipe, not HBM"}}


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


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sc = workload()
    n = sc.ncells
    times = []
    for s in range(args.warmup + args.steps):
        t, det = oracle_sample(sc, REF_SWEEPS_PER_STEP, n_sample_sweeps=10)
        if s >= args.warmup:
            times.append(t)
    t = float(np.mean(times))
    val = n / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded scene.py)",
            "config": {"workload": "random_150x150x90", "nx": 150, "ny": 150, "nz": 90,
                       "buildings": 100, "tol": 1e-6, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"per step: one single-threaded FP64 oracle step of the "
                                       f"150x150x90 workload from its initial state with 10 SOR "
                                       f"sweeps, timed phase by phase, SOR part scaled to "
                                       f"{REF_SWEEPS_PER_STEP} sweeps/step"},
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

    def timed(label, clocks_on):
        """K steps from state0, each bracketed by CUDA events on the library's
        stream after an L2 flush; max over ranks."""
        dom.set_state(state0)
        l0 = dom.timing()["launches"]
        clocks = Clocks(local) if (clocks_on and rank == 0 and not args.ncu_range) else None
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        sweeps, worst, graph_used = [], 0.0, 0
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        if args.ncu_range:
            torch.cuda.profiler.start()
        for s in range(args.steps):
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
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        if world > 1:
            ms = max_over_ranks(ms, dist, dev)
        return {"ms": ms, "sweeps": sweeps, "worst": worst, "graph": graph_used, "clocks": clk,
                "launches": launches}

    # timed region 1: the plain step (red-black SOR from the previous
    # pressure, one chunked CUDA graph per step)
    plain = timed("plain", True)
    if net is not None:
        # timed region 1b: the full hot path with the learned correction
        # (the package's network every NET_EVERY sweeps), same start state, same
        # stop test; one untimed step first builds its graphs
        dom.set_warmstart(net)
        dom.set_net_schedule(NET_EVERY)
        dom.set_state(state0)
        dom.step(1)
        learned = timed("learned", True)
        head = learned
    else:
        head = plain
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
        # the SOR kernel roofline and the CPU baseline use the plain step
        dom.set_warmstart(None)
        dom.set_state(state0)

    # timed region 2: same steps, host-driven, with CUDA events around every
    # batch of SOR sweep launches on the library's stream (kernel roofline)
    dom.set_timing(True)
    for s in range(min(args.steps, 3)):
        flush.zero_()
        dom.step(1)
    torch.cuda.synchronize()
    tm = dom.timing()
    dom.set_timing(False)

    # end to end through the C ABI with pinned host buffers (the configuration
    # of the headline value)
    if net is not None:
        dom.set_warmstart(net)
        dom.set_net_schedule(NET_EVERY)
    dom.set_state(state0)
    shapes = dom.shapes()
    host = [torch.empty(s, dtype=torch.float32, pin_memory=True).numpy() for s in shapes]
    for h, f in zip(host, dom.fields()):
        h[...] = f
    e2e_steps = max(1, min(args.steps, 3))
    h2d = sum(h.nbytes for h in host)
    torch.cuda.synchronize()
    ee = []
    for s in range(e2e_steps):
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
                                     f"every {NET_EVERY} sweeps)" if net is not None else "previous-step pressure"),
                       "l2": "flushed (256 MiB write) before every timed step"},
            "plain_sor": {"value": aggregate_mcell_steps(n, world, plain["ms"]), "unit": UNIT, "ms_per_step": plain["ms"],
                          "mean_sweeps_per_step": plain_sweeps, "max_rel_residual": plain["worst"],
                          "step_mode": "cuda_graph" if plain["graph"] else "host_loop",
                          "gpu_launches": int(plain["launches"]), "clocks": plain["clocks"]},
            "learned": None if net is None else {
                "ms_per_step": ms, "mean_sweeps_per_step": mean_sweeps,
                "speedup_vs_plain_sor": plain["ms"] / ms, "sweeps_ratio": plain_sweeps / max(mean_sweeps, 1.0),
                "net_every_sweeps": NET_EVERY, "stride": net.stride,
                "weights": os.path.relpath(WEIGHTS, ROOT),
                "note": "same start state and stop test (FP64 relative residual <= 1e-6 every step); "
                        "network time included",
                "phase_ms_per_step": net_phases},
            "roofline": {"kernel": f"{sor_kernel_name(tile)} (red-black SOR sweep, tile {les.les_sor_tile(tile) if tile >= 0 else 'two-pass'}, kc {kc})",
                         "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind,
                         "traffic": SOR_TMA_DRAM_BYTES if tile == SOR_TMA_TILE else None,
                         "bytes_per_launch": bytes_per_launch, "launch_ms": launch_ms,
                         "note": "150x150x90 SOR state (p, rhs, flags ~18 MB) is L2-resident"},
            "phase_ms_per_step": {k: tm[k] / max(tm["steps"], 1) for k in
                                  ("ms_momentum", "ms_sor", "ms_residual", "ms_project")},
            "sor_ms_per_sweep": sweep_ms,
            "gpu_launches": int(launches),
            "step_mode": "cuda_graph" if graph_used else "host_loop",
            "sor_autotune": {"tile": tile, "kc": kc, "ms_per_sweep": tune_ms},
            "e2e": {"value": aggregate_mcell_steps(n, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": h2d, "ms_per_step": e2e_ms, "steps": e2e_steps},
            "clocks": clk,
        }
        if not args.no_cpu_baseline:
            state = {"fields": [f.astype(np.float64) for f in dom.fields()],
                     "F": [dom.aux(a).astype(np.float64) for a in (les.LES_AUX_FU, les.LES_AUX_FV, les.LES_AUX_FW)],
                     "step": dom.step(0)["step"]}
            t_step, det = oracle_sample(sc, plain_sweeps, n_sample_sweeps=40, state=state)
            line["cpu_baseline"] = {
                "value": n / t_step / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": (f"one single-threaded FP64 oracle step of the same 150x150x90 state with 40 "
                           f"SOR sweeps, timed phase by phase (wall {det['sample_wall_s']:.1f} s), SOR "
                           f"part scaled to the plain GPU step's {plain_sweeps:.0f} sweeps/step (the oracle "
                           f"runs plain SOR)"),
                "detail": det}
        if not args.no_large:
            line["hbm_large"] = hbm_large(peak, peak_kind)
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="time the plain SOR step only")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the HBM-bound kernel timings on the 512x512x128 grid")
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
