"""The multi-rank host logic of bench.py on CPU: two gloo ranks, each with its
own replica timing, agree on the slowest rank's time; the whole-job value
counts every rank's sites; the reference arm prints from rank 0 only."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _rank(rank: int, world: int, port: int, out: str) -> None:
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ranks = bench.Ranks(world, "cpu")
    ranks.barrier()
    # rank r "took" 10 (r + 1) ms for its replica's steps
    ms = ranks.allmax(10.0 * (rank + 1))
    value = bench.whole_job_mlups(1000, 50, world, ms)
    ranks.barrier()
    with open(f"{out}.{rank}", "w") as fh:
        json.dump({"ms": ms, "value": value}, fh)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "rank")
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(f"{out}.{r}")) for r in range(2)]
    assert res[0] == res[1]
    assert res[0]["ms"] == 20.0
    # 2 ranks x 1000 sites x 50 steps in 20 ms
    assert res[0]["value"] == pytest.approx(2 * 1000 * 50 / 20e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    ranks = bench.Ranks(1, "cpu")
    ranks.barrier()
    assert ranks.allmax(3.5) == 3.5
    assert bench.whole_job_mlups(16777216, 200, 1, 1.6 * 200) == pytest.approx(16777216 / 1.6e-3 / 1e6)


def test_reference_arm_prints_from_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_oracle_baseline_copies_run_together():
    """The all-cores CPU baseline: independent oracle samples in child
    processes whose timed loops start together; the value counts every copy."""
    m1, dt1 = bench.oracle_in_subprocess(1, 0)
    m2, dt2 = bench.oracle_in_subprocess(1, 0, copies=2)
    sites = bench.ORACLE_SAMPLE ** 3
    assert m1 == pytest.approx(sites / dt1 / 1e6)
    assert m2 == pytest.approx(2 * sites / dt2 / 1e6)


def test_reference_arm_line():
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the keys of the benchmark contract and its own baseline and e2e."""
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == "coupled LB+Q MLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
