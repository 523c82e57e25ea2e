"""The N > 1 path of bench.py on CPU: replicas joined by a gloo process group (no
data-path collective), and the reference arm under torchrun, which rank 0 alone runs."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _replica(rank, world, port, ms, units, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.aggregate_replicas(ms[rank], units[rank], dist, "cpu")
    out.put((rank, got))
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_all_units():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    ms, units = [10.0, 12.5], [1_000_000, 3_000_000]
    procs = [ctx.Process(target=_replica, args=(r, 2, 29561, ms, units, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = (12.5, 4_000_000 / 0.0125 / 1e6)
    for r in (0, 1):
        assert res[r][0] == want[0] and abs(res[r][1] - want[1]) < 1e-9


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29563", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--config", "plain-1M-4M"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
