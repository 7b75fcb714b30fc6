"""The N-GPU bench path on CPU: two gloo ranks run bench.py's replica
aggregation (max-over-ranks time, summed solves, whole-job throughput) and
its barrier.  Replicas exchange nothing else: there is no data-path
collective in this method's single-system path."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    sys.path.insert(0, ROOT)
    import bench
    ms_local, ok_local = (100.0, 3) if rank == 0 else (150.0, 2)
    ms, ok, value = bench.replica_throughput(ms_local, ok_local, 2, torch.device("cpu"))
    bench.barrier(2)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{ms} {ok} {value}\n")
    dist.destroy_process_group()


def test_two_replicas_aggregate_like_the_bench(tmp_path):
    mp.start_processes(_rank, args=(_free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        ms, ok, value = (float(x) for x in open(tmp_path / f"rank{r}.txt").read().split())
        assert ms == 150.0 and ok == 5
        assert value == pytest.approx(5 / 0.150)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    ms, ok, value = bench.replica_throughput(80.0, 4, 1, None)
    assert (ms, ok) == (80.0, 4) and value == pytest.approx(50.0)
