"""The multi-rank path of bench.py on CPU: world_size 2 over gloo.

Ranks advance independent runs (seeds offset by rank, no data exchange) and
only the timing is reduced (max over ranks); the reference arm runs on rank 0
only."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    mem = bench.members_for_rank(rank)
    t = bench.max_over_ranks(1.5 + rank, "cpu")
    q.put((rank, mem, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing_reduction():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict()
    for _ in range(2):
        r, mem, t = q.get(timeout=120)
        out[r] = (mem, t)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    m0, m1 = out[0][0], out[1][0]
    assert [(a, b) for a, b, _ in m0] == [(a, b) for a, b, _ in m1]       # same shapes
    assert not ({s for *_, s in m0} & {s for *_, s in m1})                 # disjoint seeds
    assert out[0][1] == out[1][1] == 2.5                                    # max over ranks
    sys.path.insert(0, ROOT)
    import bench
    pts = sum(nx * ny for nx, ny, _ in m0)
    assert bench.whole_job_rate(2, pts, 10, 2.0) == 2 * pts * 10 / 2.0


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


@pytest.mark.timeout(600)
def test_reference_arm_line_on_rank_zero():
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "0"], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-500:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
