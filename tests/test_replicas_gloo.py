"""The multi-GPU path of bench.py on CPU: replicas only (the problems are
independent), so the one collective is the max of the timed region over the
ranks.  Two gloo ranks stand in for two GPUs."""
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


def _rank(rank, world, port, times, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms_max = bench.max_over_ranks(torch, dist, times[rank], "cpu")
    out.put((rank, ms_max, bench.job_mlups(world, 1000, 10, ms_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [3.5, 7.25]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest replica's time; value counts both replicas' work
    assert [r[1] for r in res] == [7.25, 7.25]
    assert res[0][2] == pytest.approx(2 * 1000 * 10 / 7.25 / 1e3)


def test_bench_without_process_group():
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, None, 4.0, "cpu") == 4.0
    assert bench.job_mlups(1, 4096 * 4096, 400, 126.8) == pytest.approx(4096 * 4096 * 400 / 126.8 / 1e3)


def test_reference_arm_under_torchrun_prints_one_line():
    # rank 0 alone runs the reference arm (the oracle on the host) and prints;
    # the other rank exits 0 without work
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
