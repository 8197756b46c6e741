"""Multi-rank host logic of bench.py on CPU over gloo (world size 2): ranks
join from the torchrun environment, each fits its own batch of the same shape
(weak scaling, no data-path collective), the whole-job figures take the
slowest rank's time and the sum of all ranks' fits, and the reference arm runs
on rank 0 alone."""
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


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import argparse
    import hashlib
    import torch.distributed as dist
    import bench
    args = argparse.Namespace(impl="svt", workload="small", events=16)
    w, r, _ = bench.dist_setup(args, backend="gloo")
    ms, units = bench.reduce_over_ranks(w, 10.0 + r, [100 * (r + 1), 7])
    _, _, batch = bench.workload(args, r)
    digest = hashlib.sha256(batch.words.tobytes()).hexdigest()
    shapes = [None] * w
    dist.all_gather_object(shapes, (batch.n_events, digest))
    bench.dist_teardown(w)
    q.put((r, w, ms, units, shapes))


def test_two_gloo_ranks_reduce_and_shard():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms, units, shapes in res:
        assert w == 2
        assert ms == 11.0                       # slowest rank
        assert units == [300, 14]               # sum over ranks
        (n0, d0), (n1, d1) = shapes
        assert n0 == n1 == 16                   # same shape on every rank
        assert d0 != d1                         # but each rank its own events


def test_reference_arm_prints_once_from_rank0():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "2", "--warmup", "1", "--workload", "small", "--events", "40"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(x) for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
