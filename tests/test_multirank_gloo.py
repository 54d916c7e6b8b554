"""The multi-GPU path of the benchmark is replicas only (no data-path
collective): each rank runs the whole workload, the ranks meet at a barrier
around the timed region, the time is the maximum over ranks and the reported
value is all ranks' work over that time.  These world-size-2 runs exercise
that host logic on the CPU with the gloo backend."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow replica
    ms = bench.max_over_ranks(local_ms, dist)
    value = bench.job_throughput(1e9, world, ms)
    dist.barrier()
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_replicas_time_is_max_over_ranks_and_value_is_whole_job():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] == pytest.approx(2e9 / 15e-3)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(100.0, 1, 1000.0) == pytest.approx(100.0)


def test_reference_arm_prints_on_rank_zero_only():
    # under torchrun every rank but 0 exits 0 without work or output
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
