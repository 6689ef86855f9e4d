"""The multi-GPU form is replicas only: every rank carves its own image and the job's throughput is
all ranks' units over the slowest rank's time. The aggregation runs here on two gloo ranks (CPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, times, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    value, total_s = bench.replica_throughput(times[rank], 480, ws, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{value} {total_s}")


def test_replica_throughput_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    times = [0.5, 0.8]   # rank 1 is the slower replica
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, times, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        value, total_s = (float(x) for x in (tmp_path / f"rank{r}.txt").read_text().split())
        assert total_s == pytest.approx(0.8)
        assert value == pytest.approx(2 * 480 / 0.8)


def test_replica_throughput_single_rank():
    import bench
    value, total_s = bench.replica_throughput(0.25, 100, 1, "cpu")
    assert total_s == 0.25 and value == pytest.approx(400.0)
