"""The N > 1 path of bench.py on CPU: world size 2 over gloo.  The bench runs
independent replicas (one factorisation per rank, no data-path collective);
the host-side pieces are the barrier around the timed region, the maximum of
the per-rank times, the per-rank seeds and rank 0 alone printing the line."""
import json
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


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    w, r, local = bench.dist_setup()
    bench.dist_barrier(w)
    m = bench.dist_max(w, float(10 * (rank + 1)))
    q.put((r, w, local, m))
    dist.destroy_process_group()


def test_barrier_and_max_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert all(o[3] == 20.0 for o in out)          # the slowest rank's time on every rank


def test_replicas_draw_different_matrices():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    w = synth.PLAIN_2000x1500
    seeds = {bench.replica_workload(w, r).seed for r in range(4)}
    assert len(seeds) == 4
    assert bench.replica_workload(w, 0).seed == w.seed


@pytest.mark.slow
def test_reference_arm_prints_on_rank_0_only():
    port = _free_port()
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--workload", "plain_2000x1500", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    procs = [subprocess.Popen(cmd, env=dict(env, RANK=str(r), LOCAL_RANK=str(r)), cwd=ROOT,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(2)]
    outs = [p.communicate(timeout=600) for p in procs]
    assert all(p.returncode == 0 for p in procs), [o[1][-2000:] for o in outs]
    lines0 = [l for l in outs[0][0].splitlines() if l.strip()]
    lines1 = [l for l in outs[1][0].splitlines() if l.strip()]
    assert len(lines0) == 1 and lines1 == []
    rec = json.loads(lines0[0])
    assert rec["impl"] == "reference" and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"


def test_sparse_replicas_draw_different_matrices():
    """The sparse workload's rank r factors the sprand draw of seed 0 + r."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    a = bench.sparse_host(bench.SPARSE["seed"])
    b = bench.sparse_host(bench.SPARSE["seed"] + 1)
    n = bench.SPARSE["n"]
    assert a[0].size == n + 1 and b[0].size == n + 1
    assert not (a[0].size == b[0].size and np.array_equal(a[1], b[1]))
