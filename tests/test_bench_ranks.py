"""bench.py's multi-process paths on CPU (gloo, world size 2): the whole-job aggregation of a
replica run and the reference arm under torchrun (rank 0 alone measures and prints)."""
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


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as td
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    # rank r: time 10 + r ms, flops 1e15 * (r + 1), executed a quarter of that
    got = bench.over_ranks(td, 10.0 + rank, 1e15 * (rank + 1), 2.5e14 * (rank + 1), torch.device("cpu"))
    td.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump(got, fh)


def test_over_ranks_takes_the_slowest_rank_and_sums_the_work(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        with open(tmp_path / f"rank{r}.json") as fh:
            ms, flops, executed = json.load(fh)
        assert ms == 11.0 and flops == 3e15 and executed == 7.5e14


def test_over_ranks_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.over_ranks(None, 5.0, 2.0, 1.0, None) == (5.0, 2.0, 1.0)


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_one_line_from_rank_zero():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--dcut", "4",
           "--cpu-slices", "1", "--warmup", "1", "--steps", "2"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["steps"] == 2
    assert out["value"] > 0 and out["e2e"]["value"] == out["value"]
    assert out["cpu_baseline"]["kind"] == "oracle"
