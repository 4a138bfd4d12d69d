"""The multi-GPU path of bench.py is replicas only: every rank advances its own
box and the only collective is the whole-job aggregation (max time over ranks,
particles summed).  Checked here on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [10.0, 20.0][rank]
        n = [100, 300][rank]
        value, ms_max = bench.job_throughput(ms, n, 5, dist)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{value} {ms_max}")
    finally:
        dist.destroy_process_group()


def test_job_throughput_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        value, ms_max = map(float, (tmp_path / f"r{r}.txt").read_text().split())
        assert ms_max == 20.0                       # the slowest rank's time
        assert value == pytest.approx(400 * 5 / 0.020)   # all particles over it


def test_job_throughput_single_process():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    value, ms = bench.job_throughput(8.0, 1000, 4, None)
    assert ms == 8.0 and value == pytest.approx(1000 * 4 / 0.008)
