"""Generated banks: templates synthesised per call into an L2-sized ring
instead of being stored.  The synthesis is the stored bank's, so every output
must equal the stored bank's bit for bit (sigma up to the order of its
floating-point sums), across chunk boundaries and bank sub-ranges."""
import numpy as np
import pytest

import oracle
from paper_1802_01685_gb300 import bf, synth

from parity import TOL, check_maxima, check_template_rows, oracle_params, run, subset

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = bf.bf_init()
    yield h
    bf.bf_destroy(h)


@pytest.fixture(scope="module")
def banks(ctx):
    # 2 x 2 x 2 x 32 x 32 = 8192 templates of 2048 samples: three synthesis
    # chunks of 24 template tiles (3072 templates), the last one partial
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0, 0.4],
                           20.0, 1000.0, 32, 32)
    stored = bf.bf_bank_create_grid(ctx, spec, 2048.0, 1.0)
    gen = bf.bf_bank_create_grid(ctx, spec, 2048.0, 1.0, bf.BF_BANK_GENERATED)
    yield spec, stored, gen
    bf.bf_bank_destroy(stored)
    bf.bf_bank_destroy(gen)


def test_generated_read_back_matches_oracle(ctx, banks):
    spec, stored, gen = banks
    p = oracle_params(spec)
    for k0, n in ((0, 3), (3070, 5), (8190, 2)):
        got = bf.bf_bank_read(gen, k0, n)
        np.testing.assert_array_equal(got, bf.bf_bank_read(stored, k0, n))
        ref = np.stack([oracle.template(int(p["track"][k]), int(p["sense"][k]), p["f_lo"][k], p["f_hi"][k],
                                        p["D"][k], 2048.0, 2048) for k in range(k0, k0 + n)])
        check_template_rows(got, {}, ref, f"rows {k0}..{k0 + n}")


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "bf16"])
def test_generated_equals_stored(ctx, banks, prec):
    spec, stored, gen = banks
    rng = np.random.default_rng(31)
    xs = [rng.standard_normal(n).astype(np.float32) for n in (2048, 6000, 9001)]
    for b0, b1 in ((0, 0), (1000, 7000), (3072, 6144), (5, 133)):
        a, am, _ = run(ctx, stored, xs, 2048.0, prec, bank_begin=b0, bank_end=b1, want_map=True)
        g, gm, _ = run(ctx, gen, xs, 2048.0, prec, bank_begin=b0, bank_end=b1, want_map=True)
        for x, y in zip(a, g):
            np.testing.assert_array_equal(y["max"], x["max"])
            np.testing.assert_array_equal(y["argmax"], x["argmax"])
            np.testing.assert_allclose(y["sigma"], x["sigma"], rtol=1e-6)
            np.testing.assert_array_equal(y["hist"], x["hist"])
            np.testing.assert_array_equal(y["map"], x["map"])
        np.testing.assert_array_equal(gm, am)


def test_generated_against_oracle(ctx, banks):
    spec, stored, gen = banks
    p = oracle_params(spec)
    x = np.random.default_rng(4).standard_normal(5000).astype(np.float32)
    idx = np.arange(3000, 3200)                                  # crosses a chunk edge
    ref = oracle.search(x, 2048.0, subset(p, idx), 2048, want_rho=True)
    g = run(ctx, gen, [x], 2048.0, "split_bf16", bank_begin=3000, bank_end=3200)[0][0]
    check_maxima(g, ref, ref["rho"], TOL["split_bf16"], "generated")


def test_serving_rejects_generated_bank(ctx, banks):
    spec, stored, gen = banks
    with pytest.raises(bf.BFError) as e:
        bf.bf_serve_submit(ctx, gen, np.zeros(4096, np.float32), 2048.0)
    assert e.value.status == bf.BF_ENOTSUP
