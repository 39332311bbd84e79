"""Search plans: one search shape captured as a CUDA graph and replayed on new
series must give what bf_correlate gives for the same inputs."""
import numpy as np
import pytest

import oracle
from paper_1802_01685_gb300 import bf, synth

from parity import TOL, check_hist, check_map, check_maxima, check_sigma, oracle_params, subset

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__
    __graft_entry__.build()
    ctx = bf.bf_init()
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0, 0.5],
                           20.0, 1000.0, 8, 12)                  # 768 templates
    bank = bf.bf_bank_create_grid(ctx, spec, 2048.0, 1.0,
                                  bf.BF_BANK_FP32 | bf.BF_BANK_SPLIT_BF16 | bf.BF_BANK_SPLIT_FP16)
    yield ctx, bank, spec
    bf.bf_bank_destroy(bank)
    bf.bf_destroy(ctx)


def outputs(res, n, want_map):
    return [bf.bf_result_copy_to_host(res, s, want_hist=True, want_map=want_map) for s in range(n)]


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "bf16", "fft_fp32", "split_fp16"])
def test_plan_replays_equal_correlate(setup, prec):
    """Three replays on new series: each replayed result equals the oracle
    within the route's tolerance, and bf_correlate on the same inputs bit for
    bit."""
    ctx, bank, spec = setup
    lens = [2048, 5000, 9000, 2049]
    opts = bf.make_opts(precision=prec, bank_begin=10, bank_end=700, want_map=True, kappa=4.0,
                        want_tails=True)
    p = subset(oracle_params(spec), np.arange(10, 700))
    tol = TOL[prec]
    plan = bf.bf_plan_create(ctx, bank, lens, 2048.0, opts)
    try:
        for run in range(3):
            rng = np.random.default_rng(100 + run)
            xs = [rng.standard_normal(n).astype(np.float32) for n in lens]
            res = bf.bf_plan_run(plan, xs)
            got = outputs(res, len(lens), True)
            got_mean = bf.bf_result_copy_mean_max(res)
            got_tails = np.sort(bf.bf_result_copy_tails(res), order=["series", "k", "tau"])
            for x, g in zip(xs, got):                # the replay itself against the oracle
                ref = oracle.search(x, 2048.0, p, 2048, want_rho=True)
                check_maxima(g, ref, ref["rho"], tol, f"plan {prec} run {run}")
                check_sigma(g, ref, tol, f"plan {prec}")
                check_hist(g["hist"], ref["max"], tol)
                check_map(g["map"], x, 2048.0, p, 2048, 4.0, tol)
            ref_h = bf.bf_correlate(ctx, bank, xs, 2048.0, opts)
            ref = outputs(ref_h, len(lens), True)
            ref_mean = bf.bf_result_copy_mean_max(ref_h)
            ref_tails = np.sort(bf.bf_result_copy_tails(ref_h), order=["series", "k", "tau"])
            bf.bf_result_destroy(ref_h)
            for g, r in zip(got, ref):
                np.testing.assert_array_equal(g["max"], r["max"])
                np.testing.assert_array_equal(g["argmax"], r["argmax"])
                np.testing.assert_allclose(g["sigma"], r["sigma"], rtol=1e-6)
                np.testing.assert_array_equal(g["hist"], r["hist"])
                np.testing.assert_array_equal(g["map"], r["map"])
            np.testing.assert_array_equal(got_mean, ref_mean)
            np.testing.assert_array_equal(got_tails, ref_tails)
    finally:
        bf.bf_plan_destroy(plan)


@pytest.mark.parametrize("prec", ["split_bf16", "fft_fp32"])
def test_plan_with_parseval_tails(setup, prec):
    """The Parseval predictor runs inside the plan's graph: each replay's
    predicted sigma matches the oracle's, and the replay equals bf_correlate
    on the same series (maxima, predicted sigma, tails at kappa sigma_k, map)
    bit for bit."""
    ctx, bank, spec = setup
    lens = [20000, 5000, 2049]
    opts = bf.make_opts(precision=prec, bank_begin=3, bank_end=500, kappa=3.5, want_tails=True,
                        want_map=True, tail_sigma=bf.BF_SIGMA_PARSEVAL)
    p = subset(oracle_params(spec), np.arange(3, 500))
    H = oracle.bank(p, 2048.0, 2048)
    plan = bf.bf_plan_create(ctx, bank, lens, 2048.0, opts)
    try:
        for run in range(2):
            rng = np.random.default_rng(300 + run)
            xs = [synth.gw_coloured(lens[0], 2048.0, rng).astype(np.float32),
                  synth.grb_lightcurve(lens[1], 2048.0, rng).astype(np.float32),
                  rng.standard_normal(lens[2]).astype(np.float32)]
            res = bf.bf_plan_run(plan, xs)
            got = outputs(res, len(lens), True)
            got_sig = [bf.bf_result_copy_sigma_pred(res, s) for s in range(len(lens))]
            got_tails = np.sort(bf.bf_result_copy_tails(res), order=["series", "k", "tau"])
            for x, sg in zip(xs, got_sig):
                np.testing.assert_allclose(sg, oracle.parseval_sigma(x, H), rtol=2e-5, atol=1e-9)
            ref_h = bf.bf_correlate(ctx, bank, xs, 2048.0, opts)
            ref = outputs(ref_h, len(lens), True)
            ref_sig = [bf.bf_result_copy_sigma_pred(ref_h, s) for s in range(len(lens))]
            ref_tails = np.sort(bf.bf_result_copy_tails(ref_h), order=["series", "k", "tau"])
            bf.bf_result_destroy(ref_h)
            assert len(ref_tails) > 0
            for g, r, gs, rs in zip(got, ref, got_sig, ref_sig):
                np.testing.assert_array_equal(gs, rs)
                np.testing.assert_array_equal(g["max"], r["max"])
                np.testing.assert_array_equal(g["argmax"], r["argmax"])
                np.testing.assert_array_equal(g["map"], r["map"])
            np.testing.assert_array_equal(got_tails, ref_tails)
    finally:
        bf.bf_plan_destroy(plan)


def test_plan_on_a_stream_and_launch_count(setup):
    ctx, bank, spec = setup
    lens = [4096, 3000]
    plan = bf.bf_plan_create(ctx, bank, lens, 2048.0, bf.make_opts())
    rng = np.random.default_rng(7)
    xs = [torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda() for n in lens]
    s = torch.cuda.Stream()
    n0 = bf.bf_kernel_launches()
    res = bf.bf_plan_run(plan, xs, s.cuda_stream)
    s.synchronize()
    # the preparation of both series (five kernels, batched over the series),
    # the correlation and the finalize kernels, all from one graph launch
    assert bf.bf_kernel_launches() - n0 >= 5 + 3
    got = outputs(res, 2, False)
    ref_h = bf.bf_correlate(ctx, bank, xs, 2048.0, bf.make_opts())
    ref = outputs(ref_h, 2, False)
    bf.bf_result_destroy(ref_h)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g["max"], r["max"])
        np.testing.assert_array_equal(g["argmax"], r["argmax"])
    # the plan owns its result: destroying it is refused, and it stays readable
    bf.bf_result_destroy(res)
    assert "belongs to a plan" in bf.load().bf_last_error().decode()
    for g, r in zip(outputs(res, 2, False), ref):
        np.testing.assert_array_equal(g["max"], r["max"])
    bf.bf_plan_destroy(plan)


def test_plan_rejects_bad_lengths(setup):
    ctx, bank, spec = setup
    with pytest.raises(bf.BFError) as e:
        bf.bf_plan_create(ctx, bank, [100], 2048.0)
    assert e.value.status == bf.BF_EINVAL
