"""bench.py's multi-GPU path on CPU: the run is `replicas only` (independent
copies of the single-GPU workload, no data-path collective), so the only
cross-rank step is the reduction of the timings. Two gloo ranks check that
every rank takes the slowest replica's time and that the whole-job value
counts all replicas' steps; the reference arm prints its line on rank 0 only."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.replica_max(local_ms[rank], dist, "cpu")
    q.put((rank, m, bench.replicas_value(world, 20, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    local_ms = [310.0, 355.5]
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, local_ms, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == max(local_ms)
        assert abs(v - 2 * 20 / (max(local_ms) * 1e-3)) < 1e-9


def test_single_process_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_max(12.5, None, "cpu") == 12.5
    assert abs(bench.replicas_value(1, 10, 12.5) - 800.0) < 1e-9


def _reference(rank: str):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="2", LOCAL_RANK=rank)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                           "--cpu-budget", "0.5"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_line_on_rank_zero_only():
    r1 = _reference("1")
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = _reference("0")
    assert r0.returncode == 0
    lines = [l for l in r0.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "steps/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
