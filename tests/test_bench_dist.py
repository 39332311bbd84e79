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


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on a bounded sample of the
    same workload and reports the same metric and unit, with a cpu_baseline
    describing the run and an e2e entry that moves no bytes; ranks other than
    0 do no work."""
    import argparse
    args = argparse.Namespace(ref_templates=1, steps=1, warmup=0)
    assert bench.run_reference(args, 1, 2, 1) is None
    line = bench.run_reference(args, 0, 1, 0)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True and line["n_gpus"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert "1 of 65536 templates" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
