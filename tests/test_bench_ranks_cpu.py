"""The multi-rank host logic of bench.py on CPU: two gloo ranks agree on the
slower rank's step time, and the reference arm does its work on rank 0 only
(the others return at once)."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        got = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")

        class A:
            config, warmup, steps, gpus = "tiny", 0, 1, world
        # non-zero ranks leave the reference arm without doing any work
        ref = bench.run_reference(A()) if rank != 0 else 0
        out[rank] = (r, w, lr, got, ref)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_step_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank, (r, w, lr, got, ref) in res.items():
        assert (r, w, lr) == (rank, world, rank)
        assert got == 15.0
        assert ref == 0


def test_single_process_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
