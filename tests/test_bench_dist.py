"""The multi-rank timing logic of bench.py (replicas: barrier + max over ranks),
run as two gloo ranks on the CPU."""

import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    from paper_2502_20049_gb300 import replicas

    dist = replicas.init("gloo")
    r, w, lr = replicas.env()
    replicas.barrier(dist)
    t = 1.0 + r  # rank 1 is the slow one
    t_max = replicas.max_over_ranks(dist, t)
    rate = replicas.aggregate_rate(100.0, w, t_max)
    out.put((r, w, lr, t_max, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_rate():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for r, w, lr, t_max, rate in res:
        assert w == 2 and lr == r
        assert t_max == 2.0
        assert rate == pytest.approx(100.0 * 2 / 2.0)


def _leaving_worker(rank, world, port, out):
    """Rank 1 leaves between steps (after the barrier, before the reduction);
    rank 0 must get an error from its next collective, not wait forever."""
    import time

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    from paper_2502_20049_gb300 import replicas

    dist = replicas.init("gloo", timeout_s=5.0)
    replicas.barrier(dist)
    if rank == 1:
        os._exit(3)  # a rank that leaves without a clean shutdown
    t0 = time.perf_counter()
    try:
        replicas.max_over_ranks(dist, 1.0)
        out.put((0, "no error"))
    except Exception as e:  # noqa: BLE001 - any collective error is the detection
        out.put((0, f"error after {time.perf_counter() - t0:.1f} s: {type(e).__name__}"))


def test_rank_that_leaves_is_detected_by_the_others():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaving_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    rank, msg = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert rank == 0 and procs[1].exitcode == 3 and procs[0].exitcode == 0
    assert msg.startswith("error after"), msg
    assert float(msg.split()[2]) < 30.0


def test_single_rank_defaults(monkeypatch):
    from paper_2502_20049_gb300 import replicas

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.env() == (0, 1, 0)
    assert replicas.init() is None
    assert replicas.max_over_ranks(None, 3.5) == 3.5


@pytest.mark.parametrize("fluid", [None, "cumulant"])
def test_reference_arm_line(fluid):
    """bench.py --impl reference times the FP64 oracle on the host (no GPU) and
    prints one JSON line with the contract's keys; --fluid selects the
    operator of the workload it samples."""
    import json
    import subprocess
    import sys

    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c2", "--steps", "1",
           "--warmup", "3"]
    if fluid:
        cmd += ["--fluid", fluid]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert ("cumulant" in line["config"]["workload"]) == (fluid == "cumulant")
