"""The host logic of bench.py on CPU: the N > 1 path with two processes over
gloo, and the roofline arithmetic of the bench line.

Multi-GPU runs of the benchmark are independent replicas (weak scaling, no
data-path collective): the only cross-rank operations are the barrier and the
max-reduce of the timed region, checked here with gloo, and the reference arm,
which rank 0 alone runs under torchrun.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = [120.0, 180.0][rank]                  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        rate = bench.job_rate(1000, world, ms_max, steps=4)
        out.put((rank, ms_max, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, ms_max, rate in res:
        assert ms_max == 180.0                      # every rank sees the slowest
        assert rate == pytest.approx(2 * 1000 / (180.0 / 4 / 1e3))


def test_single_rank_identity():
    import importlib
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    assert bench.max_over_ranks(42.0, None, None) == 42.0
    assert bench.job_rate(10, 1, 1000.0, 1) == pytest.approx(10.0)


def test_reference_arm_rank0_only_under_torchrun():
    """bench.py --impl reference under torchrun with two ranks: rank 0 prints
    one JSON line, rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--config", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="2"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def test_alu_roofline_arithmetic():
    """The roofline object of the bench line: achieved = cost-model flops /
    launch time, peak = 2 x the measured FMA rate, frac = their ratio, and the
    nominal figure from the SM count x 128 lanes x 2 x the maximum clock."""
    import bench

    class Props:
        multi_processor_count = 152

    peaks = {"ffma": {"ops_per_s": 3.86e13, "sm_mhz": 2070.0, "reasons": []}}
    r = bench.alu_roofline(4.26e12, 98.48, peaks, Props(), 2070.0)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(4.26e12 / 0.09848 / 1e12)
    assert r["peak"] == pytest.approx(77.2)
    assert r["frac"] == pytest.approx(r["achieved"] / 77.2)
    assert r["peak_nominal"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert "measured" in r["peak_basis"]


def test_cost_model_covers_every_counted_band():
    """Every band hk_count_pairs and hk_count_ring_pairs report has a cost, and
    the cheaper rules never cost more than the ones they replace."""
    import bench
    c = bench.FLOPS_PER_PAIR
    assert set(c) == {"gh1", "gh2", "gh3", "gh4", "ring8", "core"}
    assert c["gh1"] < c["gh2"] < c["gh4"] <= c["ring8"] < c["core"]
