"""The N > 1 path of bench.py on the CPU: two gloo ranks.

The build ships replicas only (one process per GPU, no data-path
collective): the whole-job figures are the slowest rank's time and the sum of
the ranks' work, and under the reference arm only rank 0 runs and prints.
"""
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
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    # rank r: r + 1 seconds, 10 (r + 1) units
    t, u = bench.rank_totals(1.0 + rank, 10 * (1 + rank), world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"t": t, "u": u}, f)


def test_rank_totals_max_time_and_summed_work_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        got = json.load(open(tmp_path / ("rank%d.json" % r)))
        assert got == {"t": 2.0, "u": 30.0}


def test_rank_totals_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_totals(1.5, 7, 1, "cpu") == (1.5, 7.0)


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
