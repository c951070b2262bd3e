"""The multi-GPU form of the benchmark runs independent replicas (the path
does not shard: every operator lives on one GPU), and the whole-job figures
combine them: the slowest rank's time, the units of all ranks.  Checked with
two gloo ranks on the CPU (the same all-reduce code bench.py runs over NCCL)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = bench.combine_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1), torch.device("cpu"))
        out[rank] = (ms, units)
    finally:
        torch.distributed.destroy_process_group()


def test_replicas_combine_max_time_and_summed_units():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (150.0, 3000)
