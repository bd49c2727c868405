"""One rank of the world-size-2 replica check (run by tests/test_replicas.py under torchrun).

Each rank stands in for one GPU's replica of the workload: it reports a different step time,
takes the slowest rank's time through bench.py's reduction over a gloo group (CPU), and writes
what it would report to $REPLICA_OUT/rank<r>.json.
"""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402

dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
t = bench.max_over_ranks(1.0 + 0.5 * rank, dist, "cpu")
dist.barrier()
with open(os.path.join(os.environ["REPLICA_OUT"], f"rank{rank}.json"), "w") as f:
    json.dump({"rank": rank, "world": world, "t": t, "value": bench.replica_value(world, 10, t)}, f)
dist.destroy_process_group()
