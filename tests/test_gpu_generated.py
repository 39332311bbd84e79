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


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "bf16", "split_fp16", "fft_fp32"])
def test_plan_on_generated_bank(ctx, banks, prec):
    """A plan on a generated bank captures its synthesis ring in the graph
    (template chunks, or their spectra, made on the auxiliary stream; three
    chunks for the direct routes here): each replay equals bf_correlate on
    the stored bank bit for bit (on the generated bank for the routes whose
    layout the stored bank lacks), and the oracle on templates around the
    chunk edges."""
    spec, stored, gen = banks
    p = oracle_params(spec)
    lens = [5000, 2049]
    b0, b1 = 7, 8000
    opts = bf.make_opts(precision=prec, bank_begin=b0, bank_end=b1, want_map=True, kappa=4.0,
                        want_tails=True)
    ref_bank = stored if prec in ("split_bf16", "fp32", "bf16") else gen
    idx = np.array([0, 1, 3064, 3065, 3066, 6136, 6137, 7992])    # chunk edges at 3065, 6137
    plan = bf.bf_plan_create(ctx, gen, lens, 2048.0, opts)
    try:
        for run_i in range(2):
            rng = np.random.default_rng(900 + run_i)
            xs = [rng.standard_normal(n).astype(np.float32) for n in lens]
            res = bf.bf_plan_run(plan, xs)
            got = [bf.bf_result_copy_to_host(res, s, want_hist=True, want_map=True) for s in range(2)]
            got_t = np.sort(bf.bf_result_copy_tails(res), order=["series", "k", "tau"])
            ref_h = bf.bf_correlate(ctx, ref_bank, xs, 2048.0, opts)
            ref = [bf.bf_result_copy_to_host(ref_h, s, want_hist=True, want_map=True) for s in range(2)]
            ref_t = np.sort(bf.bf_result_copy_tails(ref_h), order=["series", "k", "tau"])
            bf.bf_result_destroy(ref_h)
            for g, r in zip(got, ref):
                np.testing.assert_array_equal(g["max"], r["max"])
                np.testing.assert_array_equal(g["argmax"], r["argmax"])
                np.testing.assert_allclose(g["sigma"], r["sigma"], rtol=1e-6)
                np.testing.assert_array_equal(g["hist"], r["hist"])
                np.testing.assert_array_equal(g["map"], r["map"])
            np.testing.assert_array_equal(got_t, ref_t)
            for x, g in zip(xs, got):
                o = oracle.search(x, 2048.0, subset(p, idx + b0), 2048, want_rho=True)
                gs = {k: g[k][idx] for k in ("max", "argmax", "sigma")}
                check_maxima(gs, o, o["rho"], TOL[prec], f"plan {prec}")
    finally:
        bf.bf_plan_destroy(plan)


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "bf16", "split_fp16", "fft_fp32"])
def test_serving_generated_bank(ctx, banks, prec):
    """Requests on a generated bank are served with a synthesis slot of their
    own, refilled every iteration with the template tiles (or, on the FFT
    route, their spectra) that iteration correlates.  Three requests served
    together, over bank slices that take several iterations each: every
    result equals bf_correlate on the stored bank bit for bit (on the
    generated bank for the routes whose layout the stored bank lacks), and
    the oracle on sampled templates."""
    spec, stored, gen = banks
    p = oracle_params(spec)
    ref_bank = stored if prec in ("split_bf16", "fp32", "bf16") else gen
    rng = np.random.default_rng(55)
    reqs = [(rng.standard_normal(n).astype(np.float32), b0, b1)
            for n, b0, b1 in ((6000, 0, 8192), (3000, 101, 5000), (9000, 3000, 8000))]
    opts = [bf.make_opts(precision=prec, bank_begin=b0, bank_end=b1, want_map=True, kappa=4.0,
                         want_tails=True) for _, b0, b1 in reqs]
    tickets = [bf.bf_serve_submit(ctx, gen, x, 2048.0, o) for (x, _, _), o in zip(reqs, opts)]
    for t, (x, b0, b1), o in zip(tickets, reqs, opts):
        st, res = bf.bf_serve_poll(ctx, t, 120_000_000)
        assert st == bf.BF_OK
        got = bf.bf_result_copy_to_host(res, 0, want_hist=True, want_map=True)
        got_t = np.sort(bf.bf_result_copy_tails(res), order=["k", "tau"])
        bf.bf_result_destroy(res)
        ref_h = bf.bf_correlate(ctx, ref_bank, [x], 2048.0, o)
        ref = bf.bf_result_copy_to_host(ref_h, 0, want_hist=True, want_map=True)
        ref_t = np.sort(bf.bf_result_copy_tails(ref_h), order=["k", "tau"])
        bf.bf_result_destroy(ref_h)
        np.testing.assert_array_equal(got["max"], ref["max"])
        np.testing.assert_array_equal(got["argmax"], ref["argmax"])
        np.testing.assert_allclose(got["sigma"], ref["sigma"], rtol=1e-6)
        np.testing.assert_array_equal(got["hist"], ref["hist"])
        np.testing.assert_array_equal(got["map"], ref["map"])
        np.testing.assert_array_equal(got_t, ref_t)
        n = b1 - b0
        idx = np.unique(np.clip(np.array([0, 1, 3071 - b0, 3072 - b0, 6143 - b0, 6144 - b0, n - 1]), 0, n - 1))
        o_ref = oracle.search(x, 2048.0, subset(p, idx + b0), 2048, want_rho=True)
        gs = {k: got[k][idx] for k in ("max", "argmax", "sigma")}
        check_maxima(gs, o_ref, o_ref["rho"], TOL[prec], f"served {prec}")
