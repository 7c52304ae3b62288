"""bench.py's multi-rank host logic on CPU: two gloo ranks (127.0.0.1).

Under torchrun every rank advances its own replica; the timed value is the
maximum over ranks and the throughput counts every rank's units.  These run
the same helpers bench.py uses, with a gloo process group instead of NCCL.
"""
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 17.25][rank]           # per-rank timed region, ms
        ms_max = bench.aggregate_max(ms, dist)
        bench.barrier(dist, None)
        value = bench.whole_job(1000.0, ms_max, world)
        q.put((rank, ms_max, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms_max, value in got:
        assert ms_max == 17.25
        assert value == pytest.approx(2 * 1000.0 / 17.25e-3)


def test_single_process_helpers_are_identities():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_max(3.5, None) == 3.5
    assert bench.whole_job(10.0, 2.0, 1) == pytest.approx(5000.0)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_zero():
    """--impl reference with two ranks: rank 0 times the oracle and prints the
    JSON line, rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "2", "--warmup", "0", "--workload", "bar"]
    env = dict(os.environ, OMP_NUM_THREADS="2", BENCH_REFERENCE_BUDGET_S="2")
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    import json
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def test_state_based_oracle_timing_runs_whole_steps():
    # the state-based oracle reads every node's dilation, so the CPU baseline
    # of a state-based line times whole steps over all rows
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import workloads
    oracle.build()
    w = workloads.tensile_bar(8, 4, 4, steps=3)
    w.state_based = (w.bulk_modulus, 0.6 * w.bulk_modulus)
    r = bench.oracle_sample(w, oracle.micromodulus(w.bulk_modulus, w.horizon), budget_s=0.5,
                            steps=2)
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    assert r["kind"] == "oracle" and r["value"] > 0 and r["n_bonds_total"] == len(idx)
    assert 1 <= r["steps"] <= 2 and "state-based" in r["sample"]
