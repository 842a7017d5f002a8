"""The multi-rank bench path on CPU: two gloo ranks (one process each) agree on the job's
timed region, the slowest rank's time, and read their rank and world size from the
environment the launcher sets (127.0.0.1 rendezvous)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
import bench
ws, rank, lrank = bench._dist()
t = bench.job_time(1.0 + 0.25 * rank, "cpu")
dist.barrier()
print(json.dumps({"rank": rank, "world": ws, "local": lrank, "t": t}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE="2", LOCAL_RANK=str(r), REPO_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda o: o["rank"])
    assert [o["rank"] for o in outs] == [0, 1]
    assert all(o["world"] == 2 for o in outs)
    assert all(o["t"] == 1.25 for o in outs)      # the slower rank's time on both


def test_single_process_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time(3.5, "cpu") == 3.5
