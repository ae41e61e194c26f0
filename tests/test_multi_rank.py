"""Multi-process paths on the CPU (gloo, world size 2).  The spectrometer needs no exchange
between GPUs, so an N-GPU bench runs N independent replicas: the tests cover the host
logic around them, the slowest-rank timing and the whole-job rate that bench.py reports,
and the reference arm launched the way the N-GPU bench is launched (torchrun; rank 0
alone runs and prints one line, the other ranks exit 0 without output)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        t = bench.slowest(dist, times[rank])
        q.put((rank, t, bench.whole_job_rate(world, 10, 1000, t)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_whole_job_rate():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, [1.5, 2.5], q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the rate counts both ranks' samples
    assert [r[1] for r in res] == [2.5, 2.5]
    assert res[0][2] == pytest.approx(2 * 10 * 1000 / 2.5 / 1e6)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.slowest(None, 3.25) == 3.25
    assert bench.whole_job_rate(1, 4, 31981568, 0.5) == pytest.approx(4 * 31981568 / 0.5 / 1e6)


def test_reference_arm_under_torchrun():
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "3", "--ref-seconds", "2"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0 and d["unit"] == "Msample/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
