"""The control entry point that allocates no device memory.

bf_control_randomize_static() serves callers that cannot allocate device
memory where they need the time-randomised control (its sort scratch is a
fixed array in the library's device code).  It must give exactly what the
allocating bf_control_randomize() gives, call after call, although every call
reuses the array the previous call left behind.  This file is collected last.
"""
import numpy as np
import pytest

from paper_1802_01685_gb300 import bf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = bf.bf_init()
    yield h
    bf.bf_destroy(h)


def test_static_control_matches_allocating_control_twice(ctx):
    # two calls in a row: a long series, then a shorter one that must not see
    # the first call's leftovers in the shared scratch
    for n, seed in ((bf.BF_STATIC_CONTROL_MAX, 4), (262_147, 5)):
        x = torch.from_numpy(np.random.default_rng(n).standard_normal(n).astype(np.float32)).cuda()
        ref = torch.empty_like(x)
        bf.bf_control_randomize(ctx, x, seed, ref)
        out = torch.full_like(x, float("nan"))
        s = torch.cuda.current_stream()
        bf.bf_control_randomize_static(x, seed, out, s.cuda_stream)
        s.synchronize()
        assert torch.equal(out, ref), n


def test_static_control_rejects_oversize_and_host_memory(ctx):
    n = bf.BF_STATIC_CONTROL_MAX + 1
    x = torch.zeros(n, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(bf.BFError) as e:
        bf.bf_control_randomize_static(x, 1, y)
    assert e.value.status == bf.BF_EINVAL and "exceed" in str(e.value)
    xh = np.zeros(16, np.float32)
    with pytest.raises(bf.BFError) as e:
        bf.bf_control_randomize_static(xh, 1, torch.empty(16, device="cuda"))
    assert e.value.status == bf.BF_EINVAL
