"""Split-FP16 tensor-core route (BF_SPLIT_FP16): FP16 hi and lo parts of a
series scaled by a power of two chosen on the device, and of 2^8 h.

The scaling is exact, so multiplying a series by any power of two in range
leaves every output bit for bit as it was, even where plain FP16 would
overflow (|x| > 65504) or flush the samples to zero (|x| of 1e-21, the size of
gravitational-wave strain)."""
import numpy as np
import pytest

import oracle
from paper_1802_01685_gb300 import bf, synth

from parity import TOL, check_maxima, check_sigma, oracle_params, run

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
def gw(ctx):
    """A coloured GW-like series of 3 s at 4096 Hz against 256 power-law and
    linear chirps of 4096 samples (two template tiles, 8193 lags: 16 tiles of
    512 with a ragged last one of 1)."""
    fs, M = 4096.0, 4096
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0],
                           20.0, 1000.0, 8, 8)                   # 256 templates
    p = oracle_params(spec)
    rng = np.random.default_rng(77)
    x = synth.gw_coloured(12288, fs, rng)
    k, n0 = 100, 5000
    h = oracle.template(int(p["track"][k]), int(p["sense"][k]), p["f_lo"][k], p["f_hi"][k], 1.0, fs, M)
    x[n0:n0 + M] += 6.0 * np.std(x) * np.sqrt(M) / 8.0 * h
    x = x.astype(np.float32)
    ref = oracle.search(x, fs, p, M, want_rho=True)
    bank = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, bf.BF_BANK_SPLIT_BF16 | bf.BF_BANK_SPLIT_FP16)
    yield dict(fs=fs, M=M, spec=spec, p=p, x=x, ref=ref, bank=bank)
    bf.bf_bank_destroy(bank)


def dense(ctx, bank, x, fs, prec, K, L, **kw):
    rho = torch.zeros((K, L), dtype=torch.float32, device="cuda")
    outs, _, info = run(ctx, bank, [x], fs, prec, rho_out=rho, **kw)
    return rho.cpu().numpy(), outs[0], info


def test_dense_rho_and_reductions(ctx, gw):
    fs, x, ref = gw["fs"], gw["x"], gw["ref"]
    K, L = ref["rho"].shape
    rho, g, info = dense(ctx, gw["bank"], x, fs, "split_fp16", K, L)
    err = np.abs(rho.astype(np.float64) - ref["rho"]).max()
    assert err <= TOL["split_fp16"], err
    assert info.correlations == K * L
    check_maxima(g, ref, ref["rho"], TOL["split_fp16"], "split_fp16")
    check_sigma(g, ref, TOL["split_fp16"])


def test_accuracy_matches_split_bf16(ctx, gw):
    """The FP16 parts carry 22 bits of each operand against BF16's 17, yet
    what bounds both routes is the FP32 accumulation in the tensor core: on
    coloured noise (large partial sums that cancel) and on white noise the
    dense error of split-FP16 is that of split-BF16, within 25 %."""
    fs, M, p = gw["fs"], gw["M"], gw["p"]
    white = np.random.default_rng(78).standard_normal(len(gw["x"])).astype(np.float32)
    for name, x, ref in (("coloured", gw["x"], gw["ref"]),
                         ("white", white, oracle.search(white, fs, p, M, want_rho=True))):
        K, L = ref["rho"].shape
        errs = {}
        for prec in ("split_bf16", "split_fp16"):
            rho = dense(ctx, gw["bank"], x, fs, prec, K, L)[0]
            d = np.abs(rho.astype(np.float64) - ref["rho"])
            errs[prec] = (float(d.max()), float(np.sqrt((d ** 2).mean())))
        print(f"{name}: max and rms error vs the oracle: {errs}")
        assert errs["split_fp16"][0] <= TOL["split_fp16"], errs
        assert errs["split_fp16"][1] <= 1.25 * errs["split_bf16"][1], errs


@pytest.mark.parametrize("a", [-100, -70, -1, 1, 17, 60, 100])
def test_power_of_two_scaling_is_exact(ctx, gw, a):
    """x 2^a gives the same outputs bit for bit, for a from -100 (samples near
    1e-30, far below FP16's range) to 100 (near 1e30, far above it)."""
    fs, x, ref = gw["fs"], gw["x"], gw["ref"]
    K, L = ref["rho"].shape
    opts = dict(want_tails=True, kappa=4.0)
    rho0, g0, _ = dense(ctx, gw["bank"], x, fs, "split_fp16", K, L, **opts)
    xs = np.ldexp(x, a).astype(np.float32)
    assert np.array_equal(np.ldexp(xs, -a).astype(np.float32), x)      # exact in FP32
    rho1, g1, _ = dense(ctx, gw["bank"], xs, fs, "split_fp16", K, L, **opts)
    np.testing.assert_array_equal(rho1, rho0)
    for key in ("max", "argmax", "sigma", "hist"):
        np.testing.assert_array_equal(g1[key], g0[key])


def test_strain_sized_series(ctx, gw):
    """A series at 1e-21 (not a power of two) keeps split-FP16 parity with
    the oracle, which scales with it."""
    fs, M, p = gw["fs"], gw["M"], gw["p"]
    x = (gw["x"].astype(np.float64) * 1e-21).astype(np.float32)
    ref = oracle.search(x, fs, p, M, want_rho=True)
    K, L = ref["rho"].shape
    rho, g, _ = dense(ctx, gw["bank"], x, fs, "split_fp16", K, L)
    assert np.abs(rho.astype(np.float64) - ref["rho"]).max() <= TOL["split_fp16"]
    check_maxima(g, ref, ref["rho"], TOL["split_fp16"], "1e-21")


def test_generated_bank_equals_stored(ctx, gw):
    """Templates synthesised on the fly into the FP16 layout give the stored
    bank's outputs bit for bit, on a bank slice with partial tiles."""
    fs, x = gw["fs"], gw["x"]
    gen = bf.bf_bank_create_grid(ctx, gw["spec"], fs, 1.0, bf.BF_BANK_GENERATED)
    for b0, b1 in ((0, 256), (7, 201)):
        a = run(ctx, gw["bank"], [x], fs, "split_fp16", bank_begin=b0, bank_end=b1, want_tails=True)[0][0]
        b = run(ctx, gen, [x], fs, "split_fp16", bank_begin=b0, bank_end=b1, want_tails=True)[0][0]
        for key in ("max", "argmax", "sigma", "hist"):
            np.testing.assert_array_equal(a[key], b[key])
    bf.bf_bank_destroy(gen)


def test_mixed_scales_in_one_launch(ctx, gw):
    """Each series of a batch gets its own scale: a batch of the same series
    at 2^-60, 1 and 2^40, plus one of zeros, gives per series what it gives
    alone."""
    fs, x = gw["fs"], gw["x"]
    xs = [np.ldexp(x, -60).astype(np.float32), x[:7000].copy(), np.zeros(5000, np.float32),
          np.ldexp(x[3000:], 40).astype(np.float32)]
    outs = run(ctx, gw["bank"], xs, fs, "split_fp16")[0]
    for s, xi in enumerate(xs):
        alone = run(ctx, gw["bank"], [xi], fs, "split_fp16")[0][0]
        np.testing.assert_array_equal(outs[s]["max"], alone["max"])
        np.testing.assert_array_equal(outs[s]["argmax"], alone["argmax"])
    np.testing.assert_array_equal(outs[0]["max"], run(ctx, gw["bank"], [x], fs, "split_fp16")[0][0]["max"])
    assert np.all(outs[2]["max"] == 0) and np.all(outs[2]["sigma"] == 0)
