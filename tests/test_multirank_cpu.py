"""The multi-rank host logic of bench.py on CPU with two gloo ranks (the GPU runs use NCCL with one rank
per GPU; the data path has no collective: every rank advances its own copy of the instances)."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_env()
    ms = bench.reduce_max(10.0 + 5.0 * rank, w, "cpu")      # each rank's timed region
    bench.barrier(w)
    value = bench.weak_value(w, 1000, 3, ms)
    buf = io.StringIO()
    with redirect_stdout(buf):                              # the reference arm: rank 0 alone runs it
        if rank != 0:
            bench.run_reference(SimpleNamespace(workload="2d", steps=1, warmup=0, gpus=w))
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(f"{r} {w} {local} {ms} {value} {len(buf.getvalue())}\n")
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_value(tmp_path):
    world = 2
    tmp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(world)]
    for r, row in enumerate(rows):
        rank, w, local, ms, value, printed = int(row[0]), int(row[1]), int(row[2]), float(row[3]), float(row[4]), \
            int(row[5])
        assert (rank, w, local) == (r, world, r)
        assert ms == 15.0                                   # the max over ranks, on every rank
        assert value == pytest.approx(world * 1000 * 3 / 15e-3)
        assert printed == 0                                 # non-zero ranks print nothing


def test_weak_value_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.weak_value(1, 261121, 100, 1000.0) == pytest.approx(261121 * 100)
    assert bench.reduce_max(3.5, 1) == 3.5
