"""The multi-GPU path of bench.py is N independent replicas: a barrier
before and after the timed steps and the maximum of the ranks' timings.
Checked here with world size 2 on the gloo backend (CPU only)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, w, local = bench.dist_setup(world, backend="gloo")
    bench.barrier(w)
    secs = 1.0 + rank                         # the ranks' own timings
    m = bench.max_over_ranks(secs, w)
    value = bench.replica_value(100.0, 3, m, w)
    bench.barrier(w)
    out[rank] = (r, w, m, value)
    torch.distributed.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        r, w, m, value = res[rank]
        assert (r, w) == (rank, world)
        assert m == 2.0                         # max over ranks
        assert value == pytest.approx(world * 100.0 * 3 / 2.0)


def test_single_process_needs_no_group():
    import bench
    r, w, local = bench.dist_setup(1)
    assert (r, w, local) == (0, 1, 0)
    assert bench.max_over_ranks(1.5, 1) == 1.5
    assert bench.replica_value(10.0, 2, 4.0, 1) == 5.0
