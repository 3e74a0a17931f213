"""The N > 1 logic of bench.py on the CPU: two gloo ranks. Each rank owns different problems
(seeds offset by rank, same shapes: weak scaling), the job throughput is all ranks' attempts
over the slowest rank's time, and only rank 0 reports. No data-path collective exists: the
ranks exchange nothing but the timing reductions."""
from __future__ import annotations

import json
import os
import socket
import sys

import pytest

from tests.conftest import ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    r, w, _ = bench.dist_setup(None, backend="gloo")
    probs = bench.rank_problems(r, 16, 10)
    seeds = [p.seed for p in probs]
    shapes = [(p.L, p.R) for p in probs]
    gathered = [None] * w
    dist.all_gather_object(gathered, {"seeds": seeds, "shapes": shapes})
    value, total, slowest = bench.job_throughput(100.0 * (r + 1), 1.0 + r, w)
    bench.barrier(w)
    ref = bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1",
                                                "--warmup", "0", "--problems", "32"]), r, w)
    with open(os.path.join(outdir, "rank%d.json" % r), "w") as f:
        json.dump({"gathered": gathered, "value": value, "total": total, "slowest": slowest,
                   "ref": ref}, f)
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    g = res[0]["gathered"]
    assert g[0]["shapes"] == g[1]["shapes"]                      # same work per rank
    assert not set(g[0]["seeds"]) & set(g[1]["seeds"])           # different problems
    for r in res:
        assert r["total"] == 300.0 and r["slowest"] == 2.0 and r["value"] == 150.0
    assert res[0]["ref"] is not None and res[0]["ref"]["impl"] == "reference"
    assert res[1]["ref"] is None                                 # only rank 0 reports


def test_field_workload_keeps_the_shapes():
    """--field H gives the batched workload's problems the field H and nothing else: the
    same lattices, ladders and seeds as the h = 0 workload."""
    sys.path.insert(0, ROOT)
    import bench
    args = bench.parse_args(["--field", "0.1", "--streams", "2", "--quick"])
    assert args.field == 0.1 and args.streams == 2 and args.quick
    assert bench.parse_args([]).field == 0.0
    plain = bench.rank_problems(1, 24, 10)
    field = bench.rank_problems(1, 24, 10, 1, args.field)
    assert [(p.L, p.betas, p.J, p.seed) for p in plain] == [(p.L, p.betas, p.J, p.seed)
                                                           for p in field]
    assert all(p.h == 0.0 for p in plain) and all(p.h == 0.1 for p in field)
