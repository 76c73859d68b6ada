"""Multi-rank host logic of bench.py on CPU: two gloo ranks (processes) run the
barrier and the max-over-ranks reduction the bench brackets its timed region
with, and the whole-job throughput is the units of all ranks over the slowest
rank's time.  (The decode shards into independent replicas: no data-path
collective exists to test.)"""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank, world, _ = bench._dist()
dist.init_process_group("gloo")
bench._barrier(world)
m = bench._max_over_ranks(1.5 + rank, world)
print("RESULT", rank, m, flush=True)
dist.destroy_process_group()
'''


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_barrier_and_max():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    got = sorted(tuple(l.split()[1:]) for o, _ in outs for l in o.splitlines() if l.startswith("RESULT"))
    assert got == [("0", "2.5"), ("1", "2.5")]


def test_job_rate_is_weak_scaling_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 1e9 units in 500 ms (the slower rank) = 4 giga-units/s
    assert abs(bench._job_rate(1e9, 500.0, 2) - 4.0) < 1e-12
    assert abs(bench._job_rate(16777216, 1.0, 1) - 16.777216) < 1e-12
