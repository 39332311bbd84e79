"""bf_result_copy_map_cells_async: the painted cells of a time-frequency map,
written by the kernels straight into mapped page-locked host memory (or
device memory), must be exactly the nonzero cells of the dense map, in
increasing cell index, with their values bit for bit; the count is reported
in full when the capacity is smaller; arrays the device cannot address are
refused with BF_EINVAL."""
import numpy as np
import pytest

import oracle
from paper_1802_01685_gb300 import bf, synth

from parity import STORE_ALL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = bf.bf_init()
    yield h
    bf.bf_destroy(h)


def pinned(n, dtype):
    return torch.zeros(max(n, 1), dtype=dtype).pin_memory()


def cells_of(res, s, cap, device=False):
    """(count, cell indices, values) through the sparse copy."""
    dev = "cuda" if device else None
    if device:
        cell = torch.zeros(max(cap, 1), dtype=torch.int32, device=dev)
        value = torch.zeros(max(cap, 1), dtype=torch.float32, device=dev)
        count = torch.zeros(1, dtype=torch.int32, device=dev)
    else:
        cell, value, count = pinned(cap, torch.int32), pinned(cap, torch.float32), pinned(1, torch.int32)
    stream = torch.cuda.Stream()
    bf.bf_result_copy_map_cells_async(res, s, cell[:cap], value[:cap], count, stream.cuda_stream)
    stream.synchronize()
    n = int(count.cpu().numpy().view(np.uint32)[0])
    m = min(n, cap)
    return n, cell[:m].cpu().numpy().view(np.uint32).copy(), value[:m].cpu().numpy().copy()


def dense_cells(res, s):
    mp = bf.bf_result_copy_to_host(res, s, want_map=True)["map"].ravel()
    idx = np.flatnonzero(mp)
    return idx.astype(np.uint32), mp[idx]


@pytest.fixture(scope="module")
def search(ctx):
    w = synth.tiny(seed=3, n=12000, I=8, J=16)
    x, fs = w["series"][0], w["fs"]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, w["M"] / fs, STORE_ALL)
    quiet = np.zeros(6000, np.float32)
    res = bf.bf_correlate(ctx, bank, [x, quiet, x[:7000].copy()], fs,
                          bf.make_opts(precision="split_bf16", want_map=True, kappa=3.0))
    yield res, bank, w
    bf.bf_result_destroy(res)
    bf.bf_bank_destroy(bank)


@pytest.mark.parametrize("s", [0, 1, 2])
def test_cells_equal_the_dense_map(search, s):
    res = search[0]
    idx, val = dense_cells(res, s)
    n, cell, value = cells_of(res, s, cap=idx.size + 17)
    assert n == idx.size
    np.testing.assert_array_equal(cell, idx)
    np.testing.assert_array_equal(value, val)
    if s == 1:
        assert n == 0                           # a silent series paints nothing
    else:
        assert n > 0


def test_small_capacity_reports_the_full_count(search):
    res = search[0]
    idx, val = dense_cells(res, 0)
    assert idx.size > 8
    n, cell, value = cells_of(res, 0, cap=5)
    assert n == idx.size
    np.testing.assert_array_equal(cell, idx[:5])
    np.testing.assert_array_equal(value, val[:5])
    n0, cell0, _ = cells_of(res, 0, cap=0)      # the count alone
    assert n0 == idx.size and cell0.size == 0


def test_device_outputs(search):
    res = search[0]
    idx, val = dense_cells(res, 2)
    n, cell, value = cells_of(res, 2, cap=idx.size, device=True)
    assert n == idx.size
    np.testing.assert_array_equal(cell, idx)
    np.testing.assert_array_equal(value, val)


def test_unaddressable_host_memory_is_refused(search):
    res = search[0]
    cell = np.zeros(16, np.uint32)              # pageable host memory
    value = np.zeros(16, np.float32)
    count = np.zeros(1, np.uint32)
    with pytest.raises(bf.BFError) as e:
        bf.bf_result_copy_map_cells_async(res, 0, cell, value, count)
    assert e.value.status == bf.BF_EINVAL


def test_bad_arguments(search, ctx):
    res, bank, w = search
    count = pinned(1, torch.int32)
    with pytest.raises(bf.BFError):
        bf.bf_result_copy_map_cells_async(res, 3, pinned(4, torch.int32)[:4], pinned(4, torch.float32)[:4],
                                          count)
    nomap = bf.bf_correlate(ctx, bank, [w["series"][0]], w["fs"], bf.make_opts(precision="split_bf16"))
    try:
        with pytest.raises(bf.BFError) as e:
            bf.bf_result_copy_map_cells_async(nomap, 0, pinned(4, torch.int32)[:4],
                                              pinned(4, torch.float32)[:4], count)
        assert e.value.status == bf.BF_EINVAL
    finally:
        bf.bf_result_destroy(nomap)


def test_plan_result_and_oracle_map(ctx):
    """A plan's result, checked cell by cell against the oracle's map painted at
    the same threshold (cells within the tolerance of the threshold may differ)."""
    w = synth.tiny(seed=5, n=9000, I=4, J=8)
    x, fs, M = w["series"][0], w["fs"], w["M"]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, M / fs, STORE_ALL)
    kappa = 3.0
    plan = bf.bf_plan_create(ctx, bank, [len(x)], fs, bf.make_opts(precision="fp32", want_map=True, kappa=kappa))
    try:
        res = bf.bf_plan_run(plan, [x])
        idx, val = dense_cells(res, 0)
        n, cell, value = cells_of(res, 0, cap=idx.size)
        assert n == idx.size
        np.testing.assert_array_equal(cell, idx)
        np.testing.assert_array_equal(value, val)
        from parity import oracle_params
        p = oracle_params(w["grid"])
        thr = kappa / np.sqrt(M)
        tol = 2e-5
        hi = oracle.search(x, fs, p, M, thr=thr + tol, want_map=True)["map"].ravel()
        lo = oracle.search(x, fs, p, M, thr=thr - tol, want_map=True)["map"].ravel()
        dense = np.zeros_like(hi, dtype=np.float32)
        dense[cell] = value
        assert np.all(dense >= hi - tol) and np.all(dense <= lo + tol)
    finally:
        bf.bf_plan_destroy(plan)
        bf.bf_bank_destroy(bank)
