"""The multi-rank host logic of bench.py on CPU: two gloo ranks agree on the
slowest rank's time and the whole-job value; the reference arm runs on rank
0 only."""
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


def _rank(rank, ws, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = [12.5, 17.25][rank]
    ms = bench.reduce_max(local_ms, ws, "cpu")
    q.put((rank, ms, bench.job_value(ws, 512 ** 3, 100, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [17.25, 17.25]
    assert got[0][2] == got[1][2] == pytest.approx(2 * 512 ** 3 * 100 / 17.25e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max(3.0, 1, "cpu") == 3.0
    assert bench.job_value(1, 1000, 10, 1.0) == pytest.approx(10.0)


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_prints_on_rank_zero_only(rank):
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--n", "32", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    if rank:
        assert lines == []
    else:
        d = json.loads(lines[-1])
        assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
        assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_flop_model_counts_every_transform():
    """The bench's dense-FFT flop model, recounted transform by transform:
    2.5 n log2 n flops per real transform of length n; per RK stage six
    inverse and three forward real 3D transforms, each one 1D transform per
    line along each of the three axes; per x-pass launch nine x-line
    transforms per (z, y) line plus 9 flops per point for u x omega."""
    import math

    sys.path.insert(0, ROOT)
    import bench

    for n in (64, 256, 512, 1024):
        per_pt, xpass = bench.flop_model(n)
        lines_per_axis = n * n
        one_axis = lines_per_axis * 2.5 * n * math.log2(n)
        step = 4 * 9 * 3 * one_axis
        assert per_pt * n ** 3 == pytest.approx(step, rel=1e-12)
        assert xpass == pytest.approx(9 * one_axis + 9 * n ** 3, rel=1e-12)
    assert bench.flop_model(512)[0] == pytest.approx(2430.0)
