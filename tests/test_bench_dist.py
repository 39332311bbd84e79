"""The multi-GPU bench path runs independent replicas: ranks share only a
barrier and the max of their timings.  Checked here with two CPU ranks over
gloo; no GPU is involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    barrier, max_over_ranks = bench.make_dist(w, "gloo")
    barrier()
    elapsed = 100.0 + 50.0 * rank                 # the slower rank decides
    m = max_over_ranks(elapsed)
    out[rank] = (m, bench.whole_job_value(1000.0, 5, w, m))
    barrier()
    torch.distributed.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        m, v = res[rank]
        assert m == 150.0
        assert v == pytest.approx(2 * 1000.0 * 5 / 0.150)


def test_single_rank_needs_no_process_group():
    barrier, max_over_ranks = bench.make_dist(1, "gloo")
    barrier()
    assert max_over_ranks(3.5) == 3.5
    assert bench.whole_job_value(10.0, 2, 1, 1000.0) == 20.0
