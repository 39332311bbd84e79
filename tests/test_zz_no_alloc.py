"""The control entry point that allocates no device memory.

bf_control_randomize_static() serves callers that cannot allocate device
memory where they need the time-randomised control: code inside a framework
whose allocator owns all device memory, pipelines with a fixed device-memory
plan, callers under a hard cap.  Its sort scratch is a fixed array in the
library's device code.  It must give exactly what the allocating
bf_control_randomize() gives, call after call, although every call reuses the
array the previous call left behind, and after its first call on a device it
must not allocate at all.  This file is collected last.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_1802_01685_gb300 import bf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = bf.bf_init()
    yield h
    bf.bf_destroy(h)


def test_static_control_matches_allocating_control_call_after_call(ctx):
    # calls in a row with shrinking padded sort lengths (2^19, 2^19, 2^13, 2^10,
    # 1), down to sizes below one shared-memory sort chunk: a shorter call
    # must not see the longer calls' leftovers in the shared scratch
    for n, seed in ((bf.BF_STATIC_CONTROL_MAX, 4), (262_147, 5), (5000, 6), (1000, 7), (1, 8)):
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


_FRESH = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    import oracle
    from paper_1802_01685_gb300 import bf
    sizes = (bf.BF_STATIC_CONTROL_MAX, 5000, 1)
    xs = [np.random.default_rng(n).standard_normal(n).astype(np.float32) for n in sizes]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    yd = [torch.empty_like(x) for x in xd]
    one = torch.ones(1, device="cuda")
    one_out = torch.empty_like(one)
    s = torch.cuda.current_stream()
    bf.bf_control_randomize_static(one, 3, one_out, s.cuda_stream)   # the set-up call, n = 1
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for x, y, seed in zip(xd, yd, (11, 12, 13)):
        bf.bf_control_randomize_static(x, seed, y, s.cuda_stream)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    for x, y, seed in zip(xs, yd, (11, 12, 13)):
        assert np.array_equal(y.cpu().numpy(), oracle.permute(x, seed)), len(x)
    print("free", free0, free1)
    sys.exit(0 if free0 == free1 else 3)
""")


def test_static_control_allocates_nothing_after_its_first_call():
    """In a fresh process with no context: after the n = 1 set-up call, calls
    of every size leave the device's free memory unchanged, and their
    outputs equal the oracle's permutation."""
    import __graft_entry__
    __graft_entry__.build()
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", _FRESH], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stdout[-2000:], r.stderr[-2000:])
