"""Failure detection on the GPU without a fault: the bounded waits that guard
the tensor-core pipeline give up after their limit, report through the
device status word, and leave the context usable."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1802_01685_gb300 import bf, synth

from parity import TOL, check_maxima, oracle_params, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = bf.bf_init()
    yield h
    bf.bf_destroy(h)


def test_signalled_wait_returns_at_once(ctx):
    waited = bf.bf_selftest_wait(ctx, True, 200_000)
    assert 0 <= waited < 50_000


def test_unsignalled_wait_runs_out_and_the_context_survives(ctx):
    limit_us = 20_000
    w = C.c_double()
    st = bf.load().bf_selftest_wait(ctx, 0, limit_us, C.byref(w))
    assert st == bf.BF_EDEVICE
    assert limit_us <= w.value < 1_000_000          # gave up after its limit, not later
    # the status word was cleared: a signalled wait and a search succeed
    assert bf.bf_selftest_wait(ctx, True, 200_000) < 50_000
    w_ = synth.tiny(seed=4)
    fs, M = w_["fs"], w_["M"]
    x = w_["series"][0]
    bank = bf.bf_bank_create_grid(ctx, w_["grid"], fs, 1.0)
    ref = oracle.search(x, fs, oracle_params(w_["grid"]), M, want_rho=True)
    g = run(ctx, bank, [x], fs, "split_bf16")[0][0]
    check_maxima(g, ref, ref["rho"], TOL["split_bf16"], "after a timeout")
    bf.bf_bank_destroy(bank)


def test_wait_limit_out_of_range(ctx):
    for limit in (0, 1_000_001):
        with pytest.raises(bf.BFError) as e:
            bf.bf_selftest_wait(ctx, False, limit)
        assert e.value.status == bf.BF_EINVAL
