"""The multi-process path of the benchmark on CPU: two ranks over gloo.

The solve does not shard (independent replicas, no collective on the data
path); what the launcher relies on is the rank bookkeeping, the barrier and
the max-over-ranks time, and the reference arm running on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
rank, local, world = bench.dist_env()
dist.init_process_group("gloo", init_method="env://")
t = bench.max_over_ranks(1.5 + rank, world)        # each rank's step time
bench.barrier(world)
# replica throughput: units of all ranks over the slowest rank's time
value = 1000 * world / t
print(json.dumps({"rank": rank, "local": local, "world": world, "t": t, "value": value}), flush=True)
dist.destroy_process_group()
"""


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(code, world, extra_env=None, args=()):
    port = _port()
    procs = []
    for r in range(world):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code, *args], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_two_rank_barrier_and_max_time():
    outs = _run_ranks(WORKER, 2)
    lines = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(l["rank"] for l in lines) == [0, 1]
    for l in lines:
        assert l["world"] == 2 and l["t"] == 2.5          # the slower rank's time on both ranks
        assert abs(l["value"] - 800.0) < 1e-9              # 2 replicas x 1000 units / 2.5


REF = r"""
import os, sys
sys.path.insert(0, os.environ["ROOT"])
import bench
sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "square10_q4_n25"]
bench.run_reference(bench.parse())
"""


def test_reference_arm_runs_on_rank_zero_only():
    outs = _run_ranks(REF, 2)
    lines0 = [l for l in outs[0].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and outs[1].strip() == ""
    line = json.loads(lines0[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
