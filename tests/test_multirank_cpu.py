"""The N > 1 path of bench.py on CPU: world_size-2 gloo process group.

The method does not shard across GPUs in this build (independent replicas), so the only
multi-process logic is the whole-job aggregation (slowest rank's time, summed units) and the
rank-0-only reference arm; both are checked here with gloo on 127.0.0.1.
"""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:{port}", rank=int(sys.argv[1]), world_size=2)
import bench
rank = dist.get_rank()
t, u = bench.aggregate_over_ranks(elapsed_s=1.0 + rank, units=10.0 * (rank + 1))
print(json.dumps({{"rank": rank, "t": t, "u": u}}))
dist.destroy_process_group()
"""


def test_aggregate_over_two_gloo_ranks():
    port = _free_port()
    code = WORKER.format(root=ROOT, port=port)
    procs = [subprocess.Popen([sys.executable, "-c", code, str(r)], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True) for r in range(2)]
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(o.strip().splitlines()[-1])
    import json
    res = [json.loads(o) for o in outs]
    for r in res:
        assert r["t"] == 2.0          # max over ranks
        assert r["u"] == 30.0         # sum over ranks


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(1.5, 7.0) == (1.5, 7.0)


@pytest.mark.parametrize("rank", ["1"])
def test_reference_arm_nonzero_rank_exits_without_work(rank):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="2", LOCAL_RANK=rank)
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, env=env, timeout=120)
    assert res.returncode == 0
    assert res.stdout.strip() == ""
