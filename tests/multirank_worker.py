"""Rank body of tests/test_multirank.py, launched by torch.distributed.run with
the gloo backend on the CPU: the benchmark's multi-rank host logic (slowest
rank's time, whole-job throughput, per-rank replica seed); rank 0 prints one
JSON line per rank."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    try:
        ms = 10.0 + 5.0 * rank              # rank r "took" 10 + 5 r ms per step
        slowest = bench.max_over_ranks(ms, dist, "cpu")
        value = bench.aggregate_mcell_steps(1_000_000, world, slowest)
        mine = {"rank": rank, "world": world, "slowest_ms": slowest, "value": value,
                "seed": bench.replica_seed(rank)}
        every = [None] * world
        dist.all_gather_object(every, mine)
        if rank == 0:                        # one writer: the ranks' lines cannot interleave
            for d in every:
                print(json.dumps(d), flush=True)
    finally:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
