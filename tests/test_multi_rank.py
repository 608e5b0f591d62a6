"""The benchmark's multi-rank host logic on CPU (gloo, world size 2): replicas with no data-path
collective, the job's time as the slowest rank's, the whole-job rate, and the reference arm
under torchrun (rank 0 alone runs and prints; the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        mine = [0.25, 0.75][rank]                       # this rank's timed seconds
        t = bench.max_over_ranks(mine, dist, "cpu")
        out.put((rank, t, bench.job_rate(1000, 4, world, t)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [0.75, 0.75]          # every rank sees the max
    # 2 replicas x 1000 nodes x 4 steps in 0.75 s
    assert res[0][2] == pytest.approx(2 * 1000 * 4 / 0.75)
    assert bench.max_over_ranks(0.5, None, "cpu") == 0.5


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--envs", "8", "--ref-envs", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_algorithmic_work_counts():
    """The roofline numerators on a hand-countable batch: two 16x16 pads with 10 and 0 active
    nodes and one 8x8 pad with 64 (all active)."""
    from paper_2604_20295_gb300 import inputs as I
    sc = I.custom_scene([I.flat_pad(16, 16, 1.0), I.flat_pad(8, 8, 1.0)], [0, 0, 1], {},
                        [(0, 0, 0, 0, 0, 0, 1)] * 3, 1, 1)
    w = bench.algorithmic_work(sc, np.array([10, 0, 64]))
    assert w["active"] == 10 + 64 and w["passive"] == 246        # a pad without contact counts 0
    assert w["pairs"] == 246 * 10                                # passive x active, per pad
    enc = 2 * (9 * 64 + 64 * 64)
    dec = 2 * (64 * 64 + 3 * 64)
    assert w["literal_flops"] == (256 + 64) * enc + 246 * dec + 6 * 2460
    assert w["bytes_out"] == 12 * (256 * 2 + 64)


def test_oracle_single_core_rate_is_bounded_and_leaves_all_cores():
    """The bench's single-thread oracle figure runs on a few envs, and later oracle calls go
    back to every core (OpenMP keeps the last thread count it was given)."""
    from paper_2604_20295_gb300 import inputs as I
    sc = I.hand_scene(4, seed=2)
    th = I.make_params(0)
    rate, dt, nn = bench.oracle_single_core(sc, th, np.arange(2))
    assert rate > 0 and dt > 0 and nn == 2 * (5 * 512 + 2048)
    if bench.cpu_cores() > 1:
        import oracle
        omp = oracle._load()          # OpenMP's own query, found through the oracle's library
        assert omp.omp_get_max_threads() == bench.cpu_cores()


def test_cpulist_parsing_and_no_gpu_locality_without_a_gpu():
    import torch
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("") == set()
    assert bench.parse_cpulist("5") == {5}
    if not torch.cuda.is_available():
        assert bench.gpu_local_cpus(torch, 0) is None

