"""The bench's multi-rank host logic on CPU: two gloo ranks on 127.0.0.1.

Frame pairs are independent, so N ranks run N replicas (weak scaling): each
rank deblurs its own disjoint batch, the step time is the slowest rank's and
the value counts every rank's pairs.  The GPU work itself needs a GPU; what
these tests cover is the rank-dependent host side: the input shards, the
max-over-ranks reduction through gloo, the whole-job rate, and the reference
arm leaving ranks other than 0 without work.
"""
import json
import os
import socket
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402

_RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo")
local_ms = 10.0 + 5.0 * rank           # rank 1 is the slow one
mx = bench.max_over_ranks(local_ms, world)
dist.barrier()
print(json.dumps({"rank": rank, "max": mx, "seed": bench.shard_seed(rank, 60),
                  "rate": bench.job_rate(world, 60, 4, mx)}), flush=True)
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_to_the_slowest_and_count_every_rank():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_SCRIPT, str(ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    # every rank sees the slowest rank's time
    assert [d["max"] for d in outs] == [15.0, 15.0]
    # 2 ranks x 60 pairs x 4 steps over 15 ms
    assert all(abs(d["rate"] - 2 * 60 * 4 / 0.015) < 1e-6 for d in outs)
    # disjoint, adjacent seed ranges: rank 1 starts where rank 0's 60 pairs end
    assert outs[1]["seed"] - outs[0]["seed"] == 60


def test_single_rank_helpers_need_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.shard_seed(0, 60) == bench.SEED_BASE
    assert bench.job_rate(1, 60, 10, 100.0) == 6000.0


def test_reference_arm_leaves_other_ranks_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--steps", "1"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
