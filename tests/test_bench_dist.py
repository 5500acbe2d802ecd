"""The benchmark's multi-rank logic on CPU: two gloo ranks, no GPU.

A single volume does not shard, so N ranks run independent replicas of it; a
batch of volumes is split across the ranks by voxel count.  The only collectives
are a barrier and the max of the elapsed time, and the whole-job rate counts
every rank's units over the slowest rank's time.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks("gloo")
    r.barrier()
    m = r.max(10.0 + rank)          # the slowest rank's time wins
    q.put((rank, m, bench.job_rate(1e9, world, m * 1000.0)))
    r.barrier()
    r.close()


def test_two_gloo_ranks_max_and_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in out:
        assert m == 11.0
        assert abs(rate - 2e9 / 11.0 / 1e9) < 1e-12   # 2 ranks x 1e9 units / 11 s


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(5e9, 1, 1000.0) == 5.0


def test_reference_arm_prints_once_under_two_ranks():
    # rank 0 times the oracle; rank 1 exits 0 without work or output
    port = free_port()
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "rl_64x64x32", "--steps", "1", "--warmup", "0", "--gpus", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0


def test_shard_volumes_balanced_and_complete():
    sys.path.insert(0, ROOT)
    import paper_2510_14143_gb300 as cr
    from paper_2510_14143_gb300 import synth
    shapes = synth.batch_shapes()
    vox = [a * b * c for a, b, c in shapes]
    for world in (1, 2, 3, 4, 8):
        parts = cr.shard_volumes(shapes, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(shapes)))             # every volume exactly once
        loads = [sum(vox[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(vox)          # greedy balance bound
        assert parts == cr.shard_volumes(shapes, world)     # every rank computes the same split
    with pytest.raises(ValueError):
        cr.shard_volumes(shapes, 0)


def _shard_worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import paper_2510_14143_gb300 as cr
    from paper_2510_14143_gb300 import synth
    r = bench.Ranks("gloo")
    shapes = synth.batch_shapes()
    mine = cr.shard_volumes(shapes, r.world)[r.rank]
    load = float(sum(a * b * c for a, b, c in (shapes[i] for i in mine)))
    q.put((rank, mine, load, r.max(load)))
    r.barrier()
    r.close()


def test_two_gloo_ranks_split_the_batch():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, a, la, ma), (_, b, lb, mb) = out
    assert not set(a) & set(b) and len(a) + len(b) == 64    # disjoint, whole batch
    assert ma == mb == max(la, lb)                          # both ranks see the slowest share
