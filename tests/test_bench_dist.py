"""The benchmark's multi-process path on CPU (gloo, world size 2).

On a GPU node `bench.py --gpus N` runs as N replicas under torchrun, one
process per GPU, and reports the slowest rank's time; the reference arm runs
on rank 0 alone while the other ranks exit without work.  These tests cover
that host logic without a GPU:

* `max_over_ranks` over a two-rank gloo group gives every rank the
  element-wise maximum (and is the identity without a group);
* `bench.py --impl reference` under torchrun with two processes exits 0 and
  prints exactly one JSON line, from rank 0.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 5.0], dist, "cpu")
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump(got, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        assert json.load(open(tmp_path / f"r{r}.json")) == [2.0, 10.0, 5.0]


def test_max_over_ranks_without_group():
    assert bench.max_over_ranks([3, 1.5]) == [3.0, 1.5]


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1",
           "--grid", "12", "--levels", "5"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env={**os.environ, "OMP_NUM_THREADS": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["higher_is_better"] is False
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    ph = d["cpu_baseline"]["phases"]
    assert {"t_p_s", "t_f_s", "t_s_s", "n_cg"} <= set(ph) and ph["n_cg"] >= 1
    assert min(ph["t_p_s"], ph["t_f_s"], ph["t_s_s"]) > 0
    # every step is a full run of the workload; the line states how many ran
    assert d["steps"] == len(d["cpu_baseline"]["step_times_s"]) == 2 and d["warmup"] == 0
    assert d["steps_requested"] == 2 and d["warmup_requested"] == 1
    assert d["config"]["N"] == 12 ** 3 and d["config"]["levels"] == 5
