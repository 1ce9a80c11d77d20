"""The N > 1 host path of bench.py on CPU: world-size-2 gloo process groups
(one process per rank, rendezvous on 127.0.0.1). Nothing here needs a GPU: the
data path has no collective (replicas / independent problem sets), so what
multi-process runs add is the timing reduction (max over ranks for times, sum
for work), the per-rank problem sets and rank-0-only output."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=2)
    ms, work = bench.reduce_over_ranks(dist, [10.0 + rank, 100.0 * (rank + 1)], ["max", "sum"])
    out.put((rank, ms, work, bench.batch_seed(rank)))
    dist.destroy_process_group()


def test_reduction_and_per_rank_problem_sets_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [11.0, 11.0]      # max of the per-rank times
    assert [g[2] for g in got] == [300.0, 300.0]    # summed work
    assert got[0][3] != got[1][3]                    # independent problem sets


def test_reference_arm_two_ranks_prints_one_line():
    """torchrun, 2 ranks, gloo: rank 0 alone times the oracle and prints one JSON
    line; rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
