"""bench.py's N-rank path on the CPU: two `gloo` ranks on 127.0.0.1.

Every rank runs an independent replica of the workload (the path has no
exchange step), so the only cross-rank logic is host-side: the barrier on
both sides of the timed region, the maximum of the ranks' times, the
whole-job value (all ranks' cell-updates over the slowest rank's time), and
the reference arm, which rank 0 alone runs and prints."""
import json
import os
import socket
import subprocess
import sys
import time

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

WORLD = 2
CELLS = 1024 * 512


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, outdir, sleeps):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        # the timed region of bench.py: barrier, the rank's own steps, barrier
        steps = len(sleeps[rank])
        dist.barrier()
        t0 = time.perf_counter()
        for s in sleeps[rank]:
            time.sleep(s)
        own = time.perf_counter() - t0
        dist.barrier()
        total = bench.max_over_ranks(own, "cpu")
        value = bench.whole_job_value(dist.get_world_size(), CELLS, steps, total)
        # a second reduction with exact, rank-dependent inputs
        exact = bench.max_over_ranks(1.25 + 0.5 * rank, "cpu")
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump({"own": own, "total": total, "value": value, "exact": exact, "steps": steps}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo(tmp_path):
    # rank 1 is the slow replica: its time must set the job's time on both ranks
    sleeps = [[0.01, 0.01, 0.01], [0.05, 0.05, 0.05]]
    tmp.start_processes(_rank_main, args=(_free_port(), str(tmp_path), sleeps), nprocs=WORLD,
                        join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(WORLD)]
    assert r[0]["exact"] == r[1]["exact"] == 1.75
    assert r[0]["total"] == r[1]["total"] == max(r[0]["own"], r[1]["own"])
    assert r[1]["own"] > r[0]["own"]
    assert r[0]["value"] == r[1]["value"] == WORLD * CELLS * 3 / r[1]["own"]
    # the job is never credited with the fast rank's time
    assert r[0]["value"] < WORLD * CELLS * 3 / r[0]["own"]


def test_max_over_ranks_without_process_group():
    assert bench.max_over_ranks(0.123, "cpu") == 0.123
    assert bench.whole_job_value(1, CELLS, 20, 2.0) == CELLS * 10


def _bench_env(rank):
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(WORLD),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    return env


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun the reference arm runs on rank 0 only; rank 1 exits 0
    without work and prints nothing."""
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", str(WORLD), "--steps", "1", "--warmup", "3"],
                       env=_bench_env(1), capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
    assert time.perf_counter() - t0 < 60


def test_reference_arm_rank0_line_at_two_ranks():
    """Rank 0 of a two-rank reference run prints the one JSON line with the
    world size in n_gpus and the reference's own e2e block."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", str(WORLD), "--steps", "1", "--warmup", "3", "--grid", "32"],
                       env=_bench_env(0), capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == WORLD
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    # the same workload description as the GPU arm's line, key for key
    assert line["config"] == bench.config_of(bench.workload(32))
    assert "slab" in line["cpu_baseline"]["sample"]
