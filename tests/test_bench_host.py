"""bench.py host logic without a GPU: the max-over-ranks aggregation with two
gloo ranks on CPU, the launch count, the reference arm's JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_time = 0.010 * (rank + 1)              # rank 1 is the slow one
    t = torch.tensor([my_time])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    value, t_job = bench.aggregate([float(t.item())], n=1000, iters=30, world=world)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"value": value, "t": t_job}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        j = json.load(open(tmp_path / f"r{r}.json"))
        assert j["t"] == pytest.approx(0.020)                  # the slowest rank
        assert j["value"] == pytest.approx(2 * 1000 * 30 / 0.020)


def test_launch_count():
    sys.path.insert(0, ROOT)
    import bench
    # setup: reset_boxes, bbox, lattice, morton, 3 radix-sort passes, gather,
    # levels, choose_levels, 3 tiling kernels = 13; run: reset_boxes, bbox,
    # exponents, reset_run, prep, 3 per pass, finalize, collect, export
    assert bench.launches_per_step(30) == 13 + 3 + 2 + 90 + 3


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--ref-sample", "2000"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "point-iterations/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0
