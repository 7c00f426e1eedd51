"""The benchmark's multi-rank plumbing (replicas, max over ranks) on the CPU
with the gloo backend, world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    bench.dist_init(world, False)
    bench.barrier(world)
    mx = bench.reduce_max(10.0 * (rank + 1), world)
    sm = bench.reduce_sum(rank + 1, world)
    # the reference arm runs on rank 0 only; other ranks leave without work
    rc = bench.run_reference(type("A", (), {})()) if rank == 1 else None
    q.put((rank, mx, sm, rc))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_world_size_two_gloo():
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
    assert out[0][1:3] == (20.0, 3.0) and out[1][1:3] == (20.0, 3.0)
    assert out[1][3] == 0


def test_alg_bytes_formula():
    import bench
    n, nnz = 10, 100
    assert bench.alg_bytes_per_round(n, nnz, "f64") == 4 * nnz + 4 * (n + 1) + 4 * n + 24 * n + 16 * n
    assert bench.alg_bytes_per_round(n, nnz, "f32") == 4 * nnz + 4 * (n + 1) + 4 * n + 12 * n + 8 * n + 8 * n
    assert bench.alg_bytes_per_round(n, nnz, "df64") == bench.alg_bytes_per_round(n, nnz, "f64")


def test_reference_arm_json_line():
    """bench.py --impl reference times the FP64 oracle (the only reference this
    method has) and prints one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--workload", "chung_lu_10k", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GTEPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_bench_without_a_gpu_fails_loudly():
    """bench.py's own arm has no CPU fallback: without a GPU it exits non-zero
    with a message and prints no result line."""
    import subprocess
    import sys
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--steps", "1", "--warmup", "3"],
                       cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "no CPU fallback" in (r.stdout + r.stderr)
    assert not any(line.startswith("{") for line in r.stdout.splitlines())
