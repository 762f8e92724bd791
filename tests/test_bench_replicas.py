"""The multi-GPU path of bench.py runs independent replicas (no data-path collective):
its only exchange is the MAX all-reduce of the timed region, tested here with two gloo
ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRIPT = """
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank = dist.get_rank()
ms, value = bench.replica_throughput(10.0 * (rank + 1), 1000, 5, dist, "cpu")
print(json.dumps({{"rank": rank, "ms": ms, "value": value}}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_time():
    port = str(_free_port())
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=port)
        procs.append(subprocess.Popen([sys.executable, "-c", SCRIPT.format(root=ROOT)], cwd=ROOT, env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err[-2000:]
    res = [json.loads([ln for ln in out.splitlines() if ln.startswith("{")][-1]) for out, _ in outs]
    for r in res:
        assert r["ms"] == 20.0  # the slower rank's time
        assert abs(r["value"] - 2 * 1000 * 5 / 0.020) < 1e-6  # units of both ranks over that time


def test_single_process_throughput():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.replica_throughput(4.0, 250, 2)
    assert ms == 4.0 and abs(value - 250 * 2 / 0.004) < 1e-9
