"""The multi-GPU path of bench.py is replicas only (independent solves, no
data-path collective): its host logic (process group, barrier, max over ranks
of the timed region, rank-0-only reference arm) in two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    w, r, _ = bench.dist_setup()
    bench.barrier(w)
    t = bench.allmax(w, 10.0 * (r + 1))  # each rank's timed region; the line uses the slowest
    bench.run_reference(None, w, r) if r != 0 else None  # non-zero ranks leave without work
    with open(os.path.join(out, f"rank{r}.txt"), "w") as f:
        f.write(f"{w} {r} {t}\n")
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    lines = sorted(open(tmp_path / f"rank{r}.txt").read().split() for r in range(2))
    assert lines == [["2", "0", "20.0"], ["2", "1", "20.0"]]
