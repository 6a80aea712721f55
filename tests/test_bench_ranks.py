"""The multi-rank logic of bench.py on CPU: two gloo ranks, one process
each on 127.0.0.1, as torchrun launches them (one per GPU, NCCL) on a GPU
box.  Replicas only: the ranks share no data, just barriers and the
timing reductions."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
dist.barrier()
ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, device="cpu")
units = bench.sum_over_ranks(3 + rank, dist, device="cpu")
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "ms": ms, "units": units,
                  "seed": bench.rank_seed(2, rank),
                  "value": bench.job_value(units, ms)}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
               LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return env


def test_two_gloo_ranks_reduce_time_and_units():
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=_env(r, 2, port),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(2)]
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=180)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    # every rank sees the slowest rank's time and the units of all ranks
    assert [d["ms"] for d in outs] == [15.0, 15.0]
    assert [d["units"] for d in outs] == [7.0, 7.0]
    assert outs[0]["value"] == pytest.approx(7.0 / 0.015)
    # each replica draws its own content
    assert outs[0]["seed"] != outs[1]["seed"]


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1, 0) is None
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.sum_over_ranks(4, None) == 4.0
    assert bench.job_value(40, 20.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the oracle arm runs once: rank 1 exits 0 without work
    and without output."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       env=_env(1, 2, _free_port()), capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
