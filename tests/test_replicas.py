"""The multi-GPU protocol of bench.py is replicas only (the explicit step does
not shard without a halo exchange): ranks run independent copies and meet only
in barriers and a max over the timed intervals.  That host-side protocol on two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    seconds = 1.0 + rank                         # rank 1 is the slow one
    dist.barrier()
    smax = bench.max_over_ranks(seconds)
    value = bench.replica_value(1000, w, smax)
    out[rank] = (r, w, local, smax, value)
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        r, w, local, smax, value = res[rank]
        assert (r, w, local) == (rank, world, rank)
        assert smax == pytest.approx(2.0)
        assert value == pytest.approx(2 * 1000 / 2.0)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_value(10, 1, 2.0) == 5.0
