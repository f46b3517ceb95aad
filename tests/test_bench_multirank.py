"""Multi-rank host logic of bench.py on CPU: two gloo ranks (one process per
GPU in a real run) agree on the slowest rank's time and the whole-job rate,
and the reference arm prints its one JSON line from rank 0 only."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = 1.5 + rank                         # each rank timed its own K steps
    slowest = bench.reduce_max(secs, dist, "cpu")
    passthrough = bench.reduce_max(None, dist, "cpu")
    rate = bench.whole_job_rate(1000.0, world, slowest)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slowest, passthrough, rate))


def test_max_over_ranks_and_whole_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    assert [g[0] for g in got] == [0, 1]
    for _, slowest, passthrough, rate in got:
        assert slowest == 2.5 and passthrough is None
        assert rate == pytest.approx(2 * 1000.0 / 2.5)


def test_single_process_passthrough():
    import bench
    assert bench.reduce_max(3.0, None, "cpu") == 3.0
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def _reference(rank, extra=()):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
               GRIST_MESH_CACHE=os.environ.get("GRIST_MESH_CACHE", "/tmp/grist_mesh_cache"))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--ref-level", "2", *extra], capture_output=True, text=True, env=env,
                          timeout=300, cwd=ROOT)


def test_reference_arm_prints_from_rank_zero_only():
    r1 = _reference(1)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = _reference(0)
    assert r0.returncode == 0, r0.stderr[-2000:]
    lines = [l for l in r0.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "cell-level-steps/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
