"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs, element by element."""
import numpy as np
import pytest

import oracle
from paper_1802_01685_gb300 import bf, synth

from parity import (STORE_ALL, TOL, check_hist, check_map, check_maxima, check_sigma,
                    check_template_rows, oracle_params, run, subset)

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
def tiny(ctx):
    w = synth.tiny(seed=1)
    fs, M = w["fs"], w["M"]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, M / fs, STORE_ALL)
    p = oracle_params(w["grid"])
    ref = oracle.search(w["series"][0], fs, p, M, want_rho=True)
    yield w, bank, p, ref
    bf.bf_bank_destroy(bank)


# ------------------------------------------------------------------ bank

def test_bank_templates_match_oracle(ctx):
    chirps = [(bf.BF_LINEAR, bf.BF_ASC, 50.0, 1000.0, 1.0), (bf.BF_LINEAR, bf.BF_DESC, 600.0, 700.0, 0.2),
              (bf.BF_POWERLAW, bf.BF_ASC, 20.0, 1000.0, 0.2), (bf.BF_POWERLAW, bf.BF_DESC, 40.0, 400.0, 1.0),
              (bf.BF_POWERLAW, bf.BF_ASC, 999.0, 1000.0, 0.55), (bf.BF_LINEAR, bf.BF_ASC, 1.0, 2.0, 0.37),
              (bf.BF_POWERLAW, bf.BF_ASC, 2.0, 1000.0, 1.0), (bf.BF_POWERLAW, bf.BF_DESC, 30.0, 1000.0, 0.3),
              (bf.BF_LINEAR, bf.BF_BOTH, 120.0, 800.0, 1.0), (bf.BF_POWERLAW, bf.BF_BOTH, 40.0, 400.0, 0.45)]
    fs, T, M = 2048.0, 1.0, 2048
    ref = np.stack([oracle.template(c[0], c[1], c[2], c[3], c[4], fs, M) for c in chirps])
    rows = {}
    for name, storage in (("f32", bf.BF_BANK_FP32), ("bf16", bf.BF_BANK_SPLIT_BF16),
                          ("fp16", bf.BF_BANK_SPLIT_FP16)):
        bank = bf.bf_bank_create(ctx, chirps, fs, T, storage)
        rows[name] = bf.bf_bank_read(bank, 0, len(chirps))
        assert bf.bf_bank_params(bank, 1, 1)[0] == chirps[1]
        bf.bf_bank_destroy(bank)
    # FP32 rows within 2e-6 of the oracle in L2 norm (so within 2e-6 on rho
    # at any window); the split layouts are the exact splits of those rows
    check_template_rows(rows["f32"], {"bf16": rows["bf16"], "fp16": rows["fp16"]}, ref)


def test_bank_rejects_templates_longer_than_the_limit(ctx):
    with pytest.raises(bf.BFError) as e:
        bf.bf_bank_create(ctx, [(bf.BF_LINEAR, bf.BF_ASC, 50.0, 100.0, 0.5)], 40000.0, 1.0)
    assert e.value.status == bf.BF_EINVAL and "32768" in str(e.value)


def test_bank_grid_matches_oracle_grid(ctx):
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC],
                           [0.2, 0.6, 1.0], 20.0, 1000.0, 3, 5)
    bank = bf.bf_bank_create_grid(ctx, spec, 2048.0, 1.0, bf.BF_BANK_FP32)
    p = oracle_params(spec)
    K = bf.bf_bank_size(bank)
    assert K == len(p["track"]) == synth.grid_size(spec)
    got = bf.bf_bank_params(bank, 0, K)
    for k in range(K):
        assert got[k] == (p["track"][k], p["sense"][k], p["f_lo"][k], p["f_hi"][k], p["D"][k])
    bf.bf_bank_destroy(bank)


def test_bank_rejects_invalid_chirps(ctx):
    for bad in [(bf.BF_LINEAR, bf.BF_ASC, 50.0, 1024.0, 1.0),
                (bf.BF_LINEAR, bf.BF_ASC, 0.0, 100.0, 1.0),
                (bf.BF_LINEAR, bf.BF_ASC, 50.0, 100.0, 1.5),
                (3, bf.BF_ASC, 50.0, 100.0, 1.0)]:
        with pytest.raises(bf.BFError) as e:
            bf.bf_bank_create(ctx, [bad], 2048.0, 1.0)
        assert e.value.status == bf.BF_EINVAL


# ------------------------------------------------------------------ control

@pytest.mark.parametrize("n", [1, 2, 3, 1000, 2047, 2048, 2049, 65537, 262144])
def test_control_bit_exact(ctx, n):
    x = np.random.default_rng(n).standard_normal(n).astype(np.float32)
    ref = oracle.permute(x, 4)
    got = bf.bf_control_randomize(ctx, x, 4)                   # host -> host
    np.testing.assert_array_equal(got, ref)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    bf.bf_control_randomize(ctx, xd, 4, yd)                    # device -> device
    np.testing.assert_array_equal(yd.cpu().numpy(), ref)


def test_control_seed_edge_values(ctx):
    x = np.arange(5000, dtype=np.float32)
    for seed in (0, 2 ** 64 - 1, 0x9E3779B97F4A7C15):
        np.testing.assert_array_equal(bf.bf_control_randomize(ctx, x, seed), oracle.permute(x, seed))


# ------------------------------------------------------------------ tiny config, full parity

@pytest.mark.parametrize("prec,lt", [("split_bf16", 0), ("split_bf16", 256), ("fp32", 0),
                                     ("split_fp16", 0), ("split_fp16", 256),
                                     ("bf16", 512), ("bf16", 256), ("fft_fp32", 0)])
def test_tiny_dense_rho(ctx, tiny, prec, lt):
    w, bank, p, ref = tiny
    x, fs = w["series"][0], w["fs"]
    K, L = ref["rho"].shape
    rho = torch.zeros((K, L), dtype=torch.float32, device="cuda")
    outs, _, info = run(ctx, bank, [x], fs, prec, rho_out=rho, tile_lags=lt)
    if lt:
        assert info.tile_lags == lt
    elif prec.startswith("split"):
        assert info.tile_lags == 256                      # the split routes' one shape
    err = np.abs(rho.cpu().numpy().astype(np.float64) - ref["rho"])
    assert err.max() <= TOL[prec], f"{prec}: max |rho - oracle| = {err.max():.3e}"
    assert info.correlations == K * L


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "bf16", "fft_fp32", "split_fp16"])
def test_tiny_maxima_sigma_hist(ctx, tiny, prec):
    w, bank, p, ref = tiny
    x, fs = w["series"][0], w["fs"]
    outs, mean, _ = run(ctx, bank, [x], fs, prec)
    g = outs[0]
    frac = check_maxima(g, ref, ref["rho"], TOL[prec], prec)
    # the margin rule leaves fewer templates to compare at the looser BF16 bound
    assert frac > (0.3 if prec == "bf16" else 0.5)
    check_sigma(g, ref, TOL[prec], prec)
    check_hist(g["hist"], ref["max"], TOL[prec])
    np.testing.assert_array_equal(mean, g["max"])             # one series


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "fft_fp32", "split_fp16"])
def test_tiny_tf_map(ctx, tiny, prec):
    w, bank, p, ref = tiny
    x, fs, M = w["series"][0], w["fs"], w["M"]
    kappa = 3.5                                               # enough tails to paint
    outs, _, info = run(ctx, bank, [x], fs, prec, want_map=True, kappa=kappa)
    assert info.candidates_overflow == 0 and info.n_candidates > 0
    n_ref, n_gpu = check_map(outs[0]["map"], x, fs, p, M, kappa, TOL[prec])
    assert n_gpu > 0


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "bf16", "fft_fp32", "split_fp16"])
def test_tiny_tails(ctx, tiny, prec):
    """The tail list holds every (k, tau) with |rho| >= thr + tol, nothing
    below thr - tol, each with its rho within tol."""
    w, bank, p, ref = tiny
    x, fs, M = w["series"][0], w["fs"], w["M"]
    kappa, tol = 3.5, TOL[prec]
    thr = kappa / np.sqrt(M)
    res = bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts(precision=prec, want_tails=True,
                                                           kappa=kappa))
    info = bf.bf_result_info_get(res)
    tails = bf.bf_result_copy_tails(res)
    bf.bf_result_destroy(res)
    assert info.candidates_overflow == 0 and len(tails) == info.n_candidates
    a = np.abs(ref["rho"])
    got = {(int(t["k"]), int(t["tau"])): float(t["rho"]) for t in tails}
    assert len(got) == len(tails)                                 # no duplicates
    must = set(zip(*[v.tolist() for v in np.nonzero(a >= thr + tol)]))
    may = set(zip(*[v.tolist() for v in np.nonzero(a >= thr - tol)]))
    assert must <= set(got) <= may
    for (k, tau), r in got.items():
        assert abs(r - ref["rho"][k, tau]) <= tol
    assert np.all(tails["series"] == 0)
    res = bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts(precision=prec))
    with pytest.raises(bf.BFError):
        bf.bf_result_tails(res)                                   # not requested
    bf.bf_result_destroy(res)


def test_parseval_predictor_matches_oracle(ctx):
    """sigma_k predicted before the search (Parseval) against the FP64
    oracle: white noise, coloured GW-like noise, a Poisson light curve, and a
    series shorter than the 16384-sample FFT (one zero-padded segment)."""
    rng = np.random.default_rng(41)
    fs, M = 2048.0, 2048
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0, 0.35],
                           20.0, 1000.0, 4, 5)                    # 160 templates
    p = oracle_params(spec)
    H = oracle.bank(p, fs, M)
    bank = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, STORE_ALL)
    xs = [synth.white(20000, rng).astype(np.float32),
          synth.gw_coloured(30000, fs, rng).astype(np.float32),
          synth.grb_lightcurve(25000, fs, rng).astype(np.float32),
          synth.white(3000, rng).astype(np.float32)]
    for prec in ("split_bf16", "fp32", "split_fp16"):
        res = bf.bf_correlate(ctx, bank, xs, fs, bf.make_opts(precision=prec, bank_begin=7,
                                                               bank_end=150,
                                                               tail_sigma=bf.BF_SIGMA_PARSEVAL))
        for s, x in enumerate(xs):
            got = bf.bf_result_copy_sigma_pred(res, s)
            ref = oracle.parseval_sigma(x, H[7:150])
            np.testing.assert_allclose(got, ref, rtol=2e-5, atol=1e-9)
        bf.bf_result_destroy(res)
    res = bf.bf_correlate(ctx, bank, xs[:1], fs)
    with pytest.raises(bf.BFError):
        bf.bf_result_copy_sigma_pred(res, 0)                      # not requested
    bf.bf_result_destroy(res)
    bf.bf_bank_destroy(bank)


def test_parseval_predictor_long_templates_and_several_segments(ctx):
    """A 15 s series at 8192 Hz (14 Welch segments of 16384 samples at hop
    8192) and templates of 8192 samples, the longest the predictor's
    16384-point transform takes; longer templates answer BF_ENOTSUP."""
    rng = np.random.default_rng(43)
    fs = 8192.0
    chirps = [(bf.BF_LINEAR, bf.BF_ASC, 100.0, 3000.0, 1.0), (bf.BF_POWERLAW, bf.BF_DESC, 50.0, 2000.0, 0.6),
              (bf.BF_LINEAR, bf.BF_BOTH, 300.0, 900.0, 0.8)]
    bank = bf.bf_bank_create(ctx, chirps, fs, 1.0, STORE_ALL)
    p = {k: np.array([c[i] for c in chirps], dt) for i, (k, dt) in enumerate(
        (("track", np.int32), ("sense", np.int32), ("f_lo", np.float64), ("f_hi", np.float64), ("D", np.float64)))}
    x = synth.gw_coloured(int(15 * fs), fs, rng).astype(np.float32)
    res = bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts(precision="split_bf16",
                                                           tail_sigma=bf.BF_SIGMA_PARSEVAL))
    got = bf.bf_result_copy_sigma_pred(res, 0)
    bf.bf_result_destroy(res)
    np.testing.assert_allclose(got, oracle.parseval_sigma(x, oracle.bank(p, fs, 8192)), rtol=2e-5, atol=1e-9)
    bf.bf_bank_destroy(bank)
    long_bank = bf.bf_bank_create(ctx, [(bf.BF_LINEAR, bf.BF_ASC, 100.0, 3000.0, 1.0)], 16384.0, 1.0, STORE_ALL)
    with pytest.raises(bf.BFError) as e:
        bf.bf_correlate(ctx, long_bank, [np.zeros(20000, np.float32)], 16384.0,
                        bf.make_opts(tail_sigma=bf.BF_SIGMA_PARSEVAL))
    assert e.value.status == bf.BF_ENOTSUP
    bf.bf_bank_destroy(long_bank)


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "fft_fp32", "split_fp16"])
def test_parseval_tails_and_map(ctx, prec):
    """Tails |rho| >= kappa sigma_k with sigma_k predicted per template: the
    list and the map against the oracle with per-template thresholds."""
    w = synth.gw_pair(n=16384, I=8, J=8)
    fs, M = w["fs"], w["M"]
    x = w["series"][0]
    p = oracle_params(w["grid"])
    H = oracle.bank(p, fs, M)
    kappa, tol = 3.0, TOL[prec]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, STORE_ALL)
    res = bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts(
        precision=prec, kappa=kappa, want_tails=True, want_map=True,
        tail_sigma=bf.BF_SIGMA_PARSEVAL))
    sig = bf.bf_result_copy_sigma_pred(res, 0).astype(np.float64)
    tails = bf.bf_result_copy_tails(res)
    mp = bf.bf_result_copy_to_host(res, 0, want_map=True)["map"]
    bf.bf_result_destroy(res)
    ref_sig = oracle.parseval_sigma(x, H)
    np.testing.assert_allclose(sig, ref_sig, rtol=2e-5)
    thr = kappa * ref_sig
    ref = oracle.search(x, fs, p, M, want_rho=True)
    a = np.abs(ref["rho"])
    slack = tol + kappa * 2e-5 * thr                              # rho and threshold rounding
    got = {(int(t["k"]), int(t["tau"])) for t in tails}
    must = set(zip(*[v.tolist() for v in np.nonzero(a >= (thr + slack)[:, None])]))
    may = set(zip(*[v.tolist() for v in np.nonzero(a >= (thr - slack)[:, None])]))
    assert len(must) > 0 and must <= got <= may
    hi = oracle.search(x, fs, p, M, thr_k=thr + slack, want_map=True)["map"]
    lo = oracle.search(x, fs, p, M, thr_k=thr - slack, want_map=True)["map"]
    assert np.all(mp >= hi - tol) and np.all(mp <= lo + tol)
    bf.bf_bank_destroy(bank)


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "fft_fp32", "split_fp16"])
def test_butterfly_templates(ctx, prec):
    """Superposed templates (ascending + descending, both senses at once):
    dense rho, maxima and the map of their two tracks against the oracle."""
    fs, M = 2048.0, 2048
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.BOTH], [1.0, 0.5],
                           50.0, 1000.0, 4, 4)                   # 64 templates
    p = oracle_params(spec)
    rng = np.random.default_rng(52)
    x = rng.standard_normal(9000)
    h = oracle.template(int(p["track"][5]), synth.BOTH, p["f_lo"][5], p["f_hi"][5], 1.0, fs, M)
    x[2000:2000 + M] += 20.0 * h
    x = x.astype(np.float32)
    bank = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, STORE_ALL)
    ref = oracle.search(x, fs, p, M, want_rho=True)
    K, L = ref["rho"].shape
    rho = torch.zeros((K, L), dtype=torch.float32, device="cuda")
    outs, _, _ = run(ctx, bank, [x], fs, prec, rho_out=rho)
    assert np.abs(rho.cpu().numpy() - ref["rho"]).max() <= TOL[prec]
    check_maxima(outs[0], ref, ref["rho"], TOL[prec], prec)
    assert outs[0]["argmax"][5] == 2000
    outs, _, _ = run(ctx, bank, [x], fs, prec, want_map=True, kappa=4.0)
    check_map(outs[0]["map"], x, fs, p, M, 4.0, TOL[prec])
    bf.bf_bank_destroy(bank)


def test_injection_recovered(ctx):
    """A bank template injected into noise is found at its offset."""
    fs, M = 2048.0, 2048
    spec = synth.grid_spec([synth.LINEAR], [synth.ASC, synth.DESC], [1.0], 50.0, 1000.0, 4, 4)
    p = oracle_params(spec)
    k, n0 = 21, 3000
    h = oracle.template(int(p["track"][k]), int(p["sense"][k]), p["f_lo"][k], p["f_hi"][k], 1.0, fs, M)
    x = np.random.default_rng(3).standard_normal(8192)
    x[n0:n0 + M] += 30.0 * h
    x = x.astype(np.float32)
    bank = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, STORE_ALL)
    for prec in ("split_bf16", "fp32", "bf16", "split_fp16"):
        g = run(ctx, bank, [x], fs, prec)[0][0]
        assert g["argmax"][k] == n0 and g["max"][k] == g["max"].max()
    bf.bf_bank_destroy(bank)


# ------------------------------------------------------------------ ragged batch and edges

def test_ragged_batch_and_bank_slice(ctx):
    """Several series of uneven length in one launch (one exactly M long, one
    M + 1, ragged lag tiles), a bank whose size is not a multiple of the tile
    and a sub-range of it, zero windows inside a series."""
    fs, M = 1024.0, 1024
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0, 0.45],
                           20.0, 500.0, 5, 5)                    # 200 templates
    p = oracle_params(spec)
    rng = np.random.default_rng(5)
    lens = [M, M + 1, 1537, 2 * M + 700, 5000]
    xs = [rng.standard_normal(n).astype(np.float32) for n in lens]
    xs[3][100:1700] = 0.0                                        # windows of zeros
    bank = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, STORE_ALL)
    b0, b1 = 37, 181
    for prec in ("split_bf16", "fp32", "bf16", "fft_fp32", "split_fp16"):
        outs, mean, info = run(ctx, bank, xs, fs, prec, bank_begin=b0, bank_end=b1)
        assert info.n_templates == b1 - b0
        ps = subset(p, np.arange(b0, b1))
        acc = np.zeros(b1 - b0)
        for s, x in enumerate(xs):
            ref = oracle.search(x, fs, ps, M, want_rho=True)
            check_maxima(outs[s], ref, ref["rho"], TOL[prec], f"{prec} series {s}")
            check_sigma(outs[s], ref, TOL[prec])
            acc += ref["max"]
        np.testing.assert_allclose(mean, acc / len(xs), atol=TOL[prec])
    bf.bf_bank_destroy(bank)


def test_zero_series_gives_zero(ctx):
    fs, M = 1024.0, 1024
    spec = synth.grid_spec([synth.LINEAR], [synth.ASC], [1.0], 20.0, 500.0, 2, 2)
    bank = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, STORE_ALL)
    x = np.zeros(3000, np.float32)
    for prec in ("split_bf16", "fp32", "fft_fp32", "split_fp16"):
        g = run(ctx, bank, [x], fs, prec)[0][0]
        assert np.all(g["max"] == 0) and np.all(g["argmax"] == 0) and np.all(g["sigma"] == 0)
    bf.bf_bank_destroy(bank)


def test_invalid_calls(ctx, tiny):
    w, bank, _, _ = tiny
    x = w["series"][0]
    with pytest.raises(bf.BFError) as e:
        bf.bf_correlate(ctx, bank, [x[:2047]], w["fs"])          # shorter than M
    assert e.value.status == bf.BF_EINVAL
    with pytest.raises(bf.BFError):
        bf.bf_correlate(ctx, bank, [x], 4096.0)                  # wrong rate
    with pytest.raises(bf.BFError):
        bf.bf_correlate(ctx, bank, [x], w["fs"], bf.make_opts(bank_begin=10, bank_end=5))
    with pytest.raises(bf.BFError):
        bf.bf_correlate(ctx, bank, [], w["fs"])
    b32 = bf.bf_bank_create_grid(ctx, w["grid"], w["fs"], 1.0, bf.BF_BANK_FP32)
    for prec in ("split_bf16", "split_fp16"):                    # no split layout
        with pytest.raises(bf.BFError) as e:
            bf.bf_correlate(ctx, b32, [x], w["fs"], bf.make_opts(precision=prec))
        assert e.value.status == bf.BF_EINVAL
    bf.bf_bank_destroy(b32)
    for storage, prec in ((bf.BF_BANK_SPLIT_BF16, "split_fp16"), (bf.BF_BANK_SPLIT_FP16, "split_bf16"),
                          (bf.BF_BANK_SPLIT_FP16, "bf16"), (bf.BF_BANK_SPLIT_FP16, "fp32")):
        b1 = bf.bf_bank_create_grid(ctx, w["grid"], w["fs"], 1.0, storage)
        with pytest.raises(bf.BFError) as e:                     # the other split layout only
            bf.bf_correlate(ctx, b1, [x], w["fs"], bf.make_opts(precision=prec))
        assert e.value.status == bf.BF_EINVAL
        bf.bf_bank_destroy(b1)
    for storage in (32, bf.BF_BANK_GENERATED | bf.BF_BANK_SPLIT_FP16):
        with pytest.raises(bf.BFError) as e:                     # unknown or mixed storage bits
            bf.bf_bank_create_grid(ctx, w["grid"], w["fs"], 1.0, storage)
        assert e.value.status == bf.BF_EINVAL


@pytest.mark.parametrize("prec", ["split_bf16", "bf16", "split_fp16"])
def test_tile_shapes_agree(ctx, prec):
    """Plain BF16 has two tensor-core tile shapes that compute every output by
    the same MMA sequence, so maxima and argmaxes agree bit for bit; ragged
    lag tiles of either width and the autotuner's choice are covered.  The
    split routes run the 256-lag shape only (their K chunks need the second
    accumulator) and refuse 512."""
    fs = 2048.0
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0, 0.3],
                           20.0, 1000.0, 6, 7)                   # 336 templates
    bank = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, bf.BF_BANK_SPLIT_BF16 | bf.BF_BANK_SPLIT_FP16)
    rng = np.random.default_rng(12)
    xs = [rng.standard_normal(n).astype(np.float32) for n in (2048, 2048 + 255, 2048 + 700, 20000)]
    shapes = (256, 512, 0) if prec == "bf16" else (256, 0)
    res = {}
    for lt in shapes:
        outs, mean, info = run(ctx, bank, xs, fs, prec, tile_lags=lt, want_tails=True)
        assert info.tile_lags in (256, 512) and (lt == 0 or info.tile_lags == lt)
        if prec != "bf16":
            assert info.tile_lags == 256
        res[lt] = (outs, mean)
    for lt in shapes[1:]:
        for a, b in zip(res[256][0], res[lt][0]):
            np.testing.assert_array_equal(a["max"], b["max"])
            np.testing.assert_array_equal(a["argmax"], b["argmax"])
            np.testing.assert_allclose(a["sigma"], b["sigma"], rtol=1e-6)
            np.testing.assert_array_equal(a["hist"], b["hist"])
        np.testing.assert_array_equal(res[256][1], res[lt][1])
    bad = (128,) if prec == "bf16" else (128, 512)
    for lt in bad:
        with pytest.raises(bf.BFError) as e:
            run(ctx, bank, xs, fs, prec, tile_lags=lt)
        assert e.value.status == bf.BF_EINVAL
    bf.bf_bank_destroy(bank)


@pytest.mark.parametrize("M", [1024, 2048, 4096, 8192, 16384, 32768])
def test_matched_window_at_rho_one(ctx, M):
    """A bank template placed, scaled, into an otherwise zero series gives
    rho = 1 at its offset (Cauchy-Schwarz equality).
    This is the hardest case for FP32 accumulation: every partial sum of the
    window grows towards |x| |h|.  The tensor core truncates each MMA's
    addition to its accumulator, so the split routes add K in chunks of 2048
    samples and fold the chunks in the epilogue; the error stays inside the
    bound at every template length (about 1.1e-5 split-BF16, 1.5e-5
    split-FP16, where one accumulator reached 1e-4 at M = 16384)."""
    fs = float(M)
    chirps = [(bf.BF_LINEAR, bf.BF_ASC, 0.02 * fs, 0.4 * fs, 1.0),
              (bf.BF_POWERLAW, bf.BF_ASC, 0.01 * fs, 0.2 * fs, 1.0),
              (bf.BF_LINEAR, bf.BF_DESC, 0.1 * fs, 0.3 * fs, 0.8),
              (bf.BF_POWERLAW, bf.BF_BOTH, 0.02 * fs, 0.3 * fs, 1.0)]
    bank = bf.bf_bank_create(ctx, chirps, fs, 1.0, STORE_ALL)
    H = bf.bf_bank_read(bank, 0, len(chirps))
    worst = {}
    for k in range(len(chirps)):
        x = np.zeros(3 * M, np.float32)
        x[M:2 * M] = 3.0 * H[k]
        for prec in ("split_bf16", "split_fp16", "fp32"):
            g = run(ctx, bank, [x], fs, prec)[0][0]
            assert g["argmax"][k] == M, (prec, k)
            worst[prec] = max(worst.get(prec, 0.0), abs(float(g["max"][k]) - 1.0))
    print(f"M={M}: |max rho - 1| per route: {worst}")
    for prec, err in worst.items():
        assert err <= TOL[prec], (prec, err)
    bf.bf_bank_destroy(bank)


def test_async_stream_matches_sync(ctx, tiny):
    w, bank, _, ref = tiny
    x = torch.from_numpy(w["series"][0]).cuda()
    s = torch.cuda.Stream()
    res = bf.bf_correlate(ctx, bank, [x], w["fs"], bf.make_opts(stream=s.cuda_stream))
    s.synchronize()
    g = bf.bf_result_copy_to_host(res, 0)
    bf.bf_result_destroy(res)
    sync = run(ctx, bank, [w["series"][0]], w["fs"], "split_bf16")[0][0]
    np.testing.assert_array_equal(g["max"], sync["max"])
    np.testing.assert_array_equal(g["argmax"], sync["argmax"])


def test_skewnorm_fit_of_maxima(ctx):
    """The device fit of the maxima equals the oracle's fit of the same
    values, and the oracle's fit of its own maxima within the maxima's
    tolerance; data and the time-randomised control differ."""
    w = synth.gw_pair(n=16384, I=16, J=16)
    fs, M = w["fs"], w["M"]
    x = w["series"][0]
    c = bf.bf_control_randomize(ctx, x, w["control_seeds"][0])
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0)
    opts = bf.make_opts(precision="split_bf16")
    res = bf.bf_correlate(ctx, bank, [x, c], fs, opts)
    try:
        vm = [bf.bf_result_copy_to_host(res, s, want_hist=False)["max"] for s in range(2)]
        mean = bf.bf_result_copy_mean_max(res)
        for s, v in ((0, vm[0]), (1, vm[1]), (bf.BF_FIT_MEAN, mean)):
            g = bf.bf_result_fit_max(res, s)
            o = oracle.skewnorm_fit(v)
            assert g["n"] == len(v)
            for key in ("mean", "sd", "skewness"):
                assert abs(g[key] - o[key]) <= 1e-9 * max(1.0, abs(o[key])), (s, key, g[key], o[key])
            for key in ("xi", "omega", "alpha"):
                assert abs(g[key] - o[key]) <= 1e-6 * max(1.0, abs(o[key])), (s, key, g[key], o[key])
        ref = oracle.search(x, fs, oracle_params(w["grid"]), M)
        g0 = bf.bf_result_fit_max(res, 0)
        o0 = oracle.skewnorm_fit(ref["max"])
        assert abs(g0["mean"] - o0["mean"]) <= TOL["split_bf16"]
        assert abs(g0["sd"] - o0["sd"]) <= 2 * TOL["split_bf16"]
        # data and control differ markedly (the coloured noise of the data has
        # less power in the band of the templates than its white permutation)
        g1 = bf.bf_result_fit_max(res, 1)
        assert abs(g0["mean"] - g1["mean"]) > 5 * max(g0["sd"], g1["sd"]) / np.sqrt(g0["n"])
    finally:
        bf.bf_result_destroy(res)
        bf.bf_bank_destroy(bank)


def test_coincidence_pseudo_spectra(ctx):
    """Two detectors over one block with a common injected chirp, and their
    time-randomised controls: the device counts equal the oracle's counts of
    the same maps exactly, for several windows and for maps of unequal
    length."""
    w = synth.gw_pair(n=16384, I=16, J=16)
    fs = w["fs"]
    xs = w["series"]
    ctrl = [bf.bf_control_randomize(ctx, x, sd) for x, sd in zip(xs, w["control_seeds"])]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0)
    res = bf.bf_correlate(ctx, bank, xs + ctrl + [xs[1][:12000]], fs,
                          bf.make_opts(precision="split_bf16", want_map=True, kappa=4.0))
    try:
        maps = [bf.bf_result_copy_to_host(res, s, want_map=True)["map"] for s in range(5)]
        for a, b in ((0, 1), (2, 3), (0, 4)):
            for dfw, dt in ((50.0, 0), (50.0, 10), (0.0, 0), (1e6, 3)):
                g = bf.bf_result_coincidence(res, a, b, dfw, dt)
                o = oracle.coincidence(maps[a], maps[b], 4.0, dfw, dt)
                for k in g:
                    np.testing.assert_array_equal(g[k], o[k], err_msg=f"{a},{b},{dfw},{dt},{k}")
        # the chirp injected into both detectors at the same offset paints
        # coincident cells in its band (40-400 Hz)
        data = bf.bf_result_coincidence(res, 0, 1, 50.0, 0)
        assert data["coinc_a"][10:101].sum() > 0 and data["coinc_b"][10:101].sum() > 0
        with pytest.raises(bf.BFError):
            bf.bf_result_coincidence(res, 0, 5)
    finally:
        bf.bf_result_destroy(res)
    res = bf.bf_correlate(ctx, bank, xs, fs)
    with pytest.raises(bf.BFError):
        bf.bf_result_coincidence(res, 0, 1)                          # no maps
    bf.bf_result_destroy(res)
    bf.bf_bank_destroy(bank)


def test_concurrent_calls_from_threads(ctx, tiny):
    """Several host threads search through one context at once (tensor-core,
    SIMT and FFT routes, and a fit); every result equals the same call made
    alone."""
    import threading
    w, bank, _, _ = tiny
    x, fs = w["series"][0], w["fs"]
    precs = ["split_bf16", "fp32", "fft_fp32", "split_bf16"]
    alone = [run(ctx, bank, [x], fs, p)[0][0] for p in precs]
    got = [None] * len(precs)
    errors = []

    def worker(i):
        try:
            for _ in range(3):
                got[i] = run(ctx, bank, [x], fs, precs[i])[0][0]
        except Exception as e:                     # reported below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(precs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for a, g in zip(alone, got):
        np.testing.assert_array_equal(g["max"], a["max"])
        np.testing.assert_array_equal(g["argmax"], a["argmax"])
        np.testing.assert_array_equal(g["hist"], a["hist"])


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "bf16", "split_fp16"])
def test_zero_blocks_skipped_exactly(ctx, prec):
    """Templates sweeping 0.2-0.7 s of a 1 s window are zero outside their
    support, and a tile of them skips those 64-sample blocks of the K loop.
    The same templates in tiles that each also hold a full-length template
    (so every block runs) give the same outputs bit for bit, and both match
    the oracle."""
    fs, M = 2048.0, 2048
    rng = np.random.default_rng(33)

    def chirps(n, D, sense):
        f_lo = rng.uniform(20.0, 400.0, n)
        f_hi = f_lo + rng.uniform(50.0, 500.0, n)
        return [(int(rng.integers(2)), sense, float(a), float(b), D) for a, b in zip(f_lo, f_hi)]

    short = chirps(128, 0.2, bf.BF_ASC) + chirps(128, 0.45, bf.BF_DESC) + chirps(50, 0.7, bf.BF_BOTH)
    full = (bf.BF_LINEAR, bf.BF_ASC, 100.0, 900.0, 1.0)
    mixed, where = [], []
    for i, c in enumerate(short):
        if len(mixed) % 128 == 0:
            mixed.append(full)
        where.append(len(mixed))
        mixed.append(c)
    x = rng.standard_normal(7000)
    x[3000:3000 + M] += 25.0 * oracle.template(*short[140], fs, M)
    x = x.astype(np.float32)
    a_bank = bf.bf_bank_create(ctx, short, fs, 1.0, STORE_ALL)
    b_bank = bf.bf_bank_create(ctx, mixed, fs, 1.0, STORE_ALL)
    a = run(ctx, a_bank, [x], fs, prec, want_tails=True)[0][0]
    b = run(ctx, b_bank, [x], fs, prec, want_tails=True)[0][0]
    for key in ("max", "argmax", "sigma"):
        np.testing.assert_array_equal(a[key], b[key][where])
    p = {k: np.array([c[i] for c in short], dt)
         for i, (k, dt) in enumerate((("track", np.int32), ("sense", np.int32), ("f_lo", np.float64),
                                      ("f_hi", np.float64), ("D", np.float64)))}
    ref = oracle.search(x, fs, p, M, want_rho=True)
    check_maxima(a, ref, ref["rho"], TOL[prec], prec)
    assert a["argmax"][140] == 3000
    bf.bf_bank_destroy(a_bank)
    bf.bf_bank_destroy(b_bank)


def test_copy_into_caller_buffers(ctx, tiny):
    """Results copied into caller-owned (pinned) host arrays equal the
    default copy; arrays of the wrong shape or dtype are refused."""
    w, bank, _, _ = tiny
    x, fs = w["series"][0], w["fs"]
    res = bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts(want_map=True))
    ref = bf.bf_result_copy_to_host(res, 0, want_hist=True, want_map=True)
    K, nb = len(ref["max"]), len(ref["hist"])
    out = {"max": torch.full((K,), -1.0, pin_memory=True).numpy(),
           "argmax": torch.full((K,), -1, dtype=torch.int32, pin_memory=True).numpy(),
           "sigma": torch.zeros(K, pin_memory=True).numpy(),
           "hist": torch.zeros(nb, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32),
           "map": torch.zeros(ref["map"].shape, pin_memory=True).numpy()}
    for _ in range(2):                                           # reused across calls
        got = bf.bf_result_copy_to_host(res, 0, want_hist=True, want_map=True, out=out)
        for key in ref:
            assert got[key] is out[key]
            np.testing.assert_array_equal(got[key], ref[key])
    with pytest.raises(ValueError):
        bf.bf_result_copy_to_host(res, 0, out={"max": np.zeros(K + 1, np.float32)})
    with pytest.raises(ValueError):
        bf.bf_result_copy_to_host(res, 0, out={"argmax": np.zeros(K, np.int64)})
    bf.bf_result_destroy(res)


@pytest.mark.parametrize("prec", ["split_bf16", "fft_fp32", "fp32"])
def test_non_finite_samples_are_refused(ctx, tiny, prec):
    """A NaN or an infinity anywhere in a series makes a synchronous search
    return BF_EINVAL naming the series (host and device inputs), with no
    result; the context then runs a finite search as before."""
    w, bank, _, _ = tiny
    x, fs = w["series"][0], w["fs"]
    opts = bf.make_opts(precision=prec)
    ref = bf.bf_correlate(ctx, bank, [x], fs, opts)
    want = bf.bf_result_copy_to_host(res=ref, s=0)
    bf.bf_result_destroy(ref)
    for bad, at in ((np.nan, 3000), (np.inf, 0), (-np.inf, len(x) - 1)):
        y = x.copy()
        y[at] = bad
        for arg in (y, torch.from_numpy(y).cuda()):
            with pytest.raises(bf.BFError) as e:
                bf.bf_correlate(ctx, bank, [x, arg], fs, opts)
            assert e.value.status == bf.BF_EINVAL and "series 1" in str(e.value), str(e.value)
    res = bf.bf_correlate(ctx, bank, [x], fs, opts)
    got = bf.bf_result_copy_to_host(res, 0)
    bf.bf_result_destroy(res)
    for key in ("max", "argmax", "sigma", "hist"):
        np.testing.assert_array_equal(got[key], want[key])


@pytest.mark.parametrize("prec", ["split_bf16", "fft_fp32"])
def test_non_finite_samples_on_asynchronous_paths(ctx, tiny, prec):
    """A series holding a NaN through a call on a stream, a plan (run
    synchronously and on a stream) and a served request: the calls on a
    stream report BF_EINVAL through bf_result_check once the stream has
    synchronised, the synchronous plan run returns it, and the served request
    fails with it.  Finite series before and after check clean, on the same
    plan and context."""
    w, bank, _, _ = tiny
    x, fs = w["series"][0], w["fs"]
    y = x.copy()
    y[3000] = np.nan
    s = torch.cuda.Stream()
    for series, bad in (([x, y], True), ([x, x], False)):
        res = bf.bf_correlate(ctx, bank, series, fs, bf.make_opts(precision=prec, stream=s.cuda_stream))
        s.synchronize()
        if bad:
            with pytest.raises(bf.BFError) as e:
                bf.bf_result_check(res)
            assert e.value.status == bf.BF_EINVAL and "non-finite" in str(e.value)
        else:
            bf.bf_result_check(res)
        bf.bf_result_destroy(res)
    plan = bf.bf_plan_create(ctx, bank, [len(x), len(x)], fs, bf.make_opts(precision=prec))
    try:
        with pytest.raises(bf.BFError) as e:
            bf.bf_plan_run(plan, [x, y])
        assert e.value.status == bf.BF_EINVAL
        bf.bf_result_check(bf.bf_plan_run(plan, [x, x]))
        for series, bad in (([y, x], True), ([x, x], False)):
            res = bf.bf_plan_run(plan, series, s.cuda_stream)
            s.synchronize()
            if bad:
                with pytest.raises(bf.BFError) as e:
                    bf.bf_result_check(res)
                assert e.value.status == bf.BF_EINVAL
            else:
                bf.bf_result_check(res)
    finally:
        bf.bf_plan_destroy(plan)
    t_bad = bf.bf_serve_submit(ctx, bank, y, fs, bf.make_opts(precision=prec))
    t_good = bf.bf_serve_submit(ctx, bank, x, fs, bf.make_opts(precision=prec))
    with pytest.raises(bf.BFError) as e:
        bf.bf_serve_poll(ctx, t_bad, 60_000_000)
    assert e.value.status == bf.BF_EINVAL and "non-finite" in str(e.value)
    st, res = bf.bf_serve_poll(ctx, t_good, 60_000_000)
    assert st == bf.BF_OK
    bf.bf_result_check(res)
    bf.bf_result_destroy(res)


def test_async_copy_into_pinned_buffers(ctx, tiny):
    """bf_result_copy_to_host_async gives, once its stream is synchronised,
    what the synchronous copy gives, for every series of a batch, on a caller
    stream busy with other work first, and on the default stream. Without every array in `out`, or with a histogram that
    was not requested, it is refused before anything is enqueued."""
    w, bank, _, _ = tiny
    fs = w["fs"]
    xs = [w["series"][0], w["series"][0][:5000].copy(), w["series"][0][1000:].copy()]
    res = bf.bf_correlate(ctx, bank, xs, fs, bf.make_opts(want_map=True))
    stream = torch.cuda.Stream()
    big = torch.zeros(1 << 26, device="cuda")
    for st in (stream, None):
        refs, outs = [], []
        for s in range(len(xs)):
            ref = bf.bf_result_copy_to_host(res, s, want_hist=True, want_map=True)
            K, nb = len(ref["max"]), len(ref["hist"])
            outs.append({"max": torch.full((K,), -1.0, pin_memory=True).numpy(),
                         "argmax": torch.full((K,), -1, dtype=torch.int32, pin_memory=True).numpy(),
                         "sigma": torch.zeros(K, pin_memory=True).numpy(),
                         "hist": torch.zeros(nb, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32),
                         "map": torch.zeros(ref["map"].shape, pin_memory=True).numpy()})
            refs.append(ref)
        if st is not None:
            with torch.cuda.stream(st):
                big.mul_(2.0).add_(1.0)                      # the stream is busy first
        for s in range(len(xs)):
            got = bf.bf_result_copy_to_host_async(res, s, outs[s], st.cuda_stream if st else None,
                                                  want_hist=True, want_map=True)
            assert all(got[k] is outs[s][k] for k in got)
        if st is not None:
            st.synchronize()
        else:
            torch.cuda.default_stream().synchronize()
        for ref, out in zip(refs, outs):
            for key in ref:
                np.testing.assert_array_equal(out[key], ref[key])
    K = len(refs[0]["max"])
    with pytest.raises(ValueError):
        bf.bf_result_copy_to_host_async(res, 0, {"max": np.zeros(K, np.float32)}, want_hist=False)
    res2 = bf.bf_correlate(ctx, bank, xs[:1], fs, bf.make_opts(want_hist=False))
    o = {"max": np.zeros(K, np.float32), "argmax": np.zeros(K, np.int32), "sigma": np.zeros(K, np.float32),
         "hist": np.zeros(1024, np.uint32)}
    with pytest.raises(bf.BFError) as e:
        bf.bf_result_copy_to_host_async(res2, 0, o, want_hist=True)
    assert e.value.status == bf.BF_EINVAL
    bf.bf_result_destroy(res2)
    bf.bf_result_destroy(res)


def test_zero_blocks_skipped_quadrature_generated_ragged_m(ctx):
    """Skipping with quadrature pairs, a generated bank and M = 2000 (padded to
    2048): short-sweep templates in a generated quadrature bank give, bit for
    bit, what the same templates give in a stored bank whose tiles each hold a
    full-length chirp, and match the oracle's phase-blind output."""
    fs, M = 2000.0, 2000
    rng = np.random.default_rng(34)
    f_lo = rng.uniform(20.0, 300.0, 150)
    short = [(int(i % 2), int(i % 3), float(a), float(a + rng.uniform(60.0, 600.0)), [0.25, 0.6][i >= 64])
             for i, a in enumerate(f_lo)]
    full = (bf.BF_POWERLAW, bf.BF_ASC, 40.0, 500.0, 1.0)
    mixed, where = [], []
    for c in short:
        if len(mixed) % 64 == 0:                      # 64 chirps = 128 rows per tile
            mixed.append(full)
        where.append(len(mixed))
        mixed.append(c)
    x = rng.standard_normal(6100)
    x[2500:2500 + M] += 20.0 * oracle.template(*short[100], fs, M, 1)
    x = x.astype(np.float32)
    gen = bf.bf_bank_create(ctx, short, fs, 1.0, bf.BF_BANK_GENERATED | bf.BF_BANK_QUADRATURE)
    ref_bank = bf.bf_bank_create(ctx, mixed, fs, 1.0, bf.BF_BANK_SPLIT_BF16 | bf.BF_BANK_QUADRATURE)
    a = run(ctx, gen, [x], fs, "split_bf16")[0][0]
    b = run(ctx, ref_bank, [x], fs, "split_bf16")[0][0]
    for key in ("max", "argmax", "sigma"):
        np.testing.assert_array_equal(a[key], b[key][where])
    p = {k: np.array([c[i] for c in short], dt)
         for i, (k, dt) in enumerate((("track", np.int32), ("sense", np.int32), ("f_lo", np.float64),
                                      ("f_hi", np.float64), ("D", np.float64)))}
    ref = oracle.search(x, fs, p, M, want_rho=True, quadrature=True)
    check_maxima(a, ref, ref["rho"], TOL["split_bf16"], "quadrature skip")
    assert abs(int(a["argmax"][100]) - 2500) <= 2
    bf.bf_bank_destroy(gen)
    bf.bf_bank_destroy(ref_bank)


@pytest.mark.parametrize("scale", [1e-3, 1e-6])
def test_quiet_stretch_after_loud_data(ctx, scale):
    """Noise with a long stretch `scale` times quieter than what precedes it.
    Inside the stretch rho is normalised noise again, but the window energy is
    a tiny difference of the FP64 prefix of x^2, which those windows sum
    directly; every route matches the oracle's dense rho there."""
    fs, M = 2048.0, 2048
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0, 0.4],
                           40.0, 900.0, 4, 4)                    # 128 templates
    bank = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, STORE_ALL)
    p = oracle_params(spec)
    rng = np.random.default_rng(81)
    x = rng.standard_normal(13000)
    x[4000:9500] *= scale
    x = x.astype(np.float32)
    ref = oracle.search(x, fs, p, M, want_rho=True)
    K, L = ref["rho"].shape
    for prec in ("split_bf16", "fp32", "split_fp16", "fft_fp32", "bf16"):
        rho = torch.zeros((K, L), dtype=torch.float32, device="cuda")
        outs, _, _ = run(ctx, bank, [x], fs, prec, rho_out=rho)
        err = np.abs(rho.cpu().numpy().astype(np.float64) - ref["rho"])
        assert err.max() <= TOL[prec], (prec, err.max(), np.unravel_index(err.argmax(), err.shape))
        check_maxima(outs[0], ref, ref["rho"], TOL[prec], prec)
        check_sigma(outs[0], ref, TOL[prec])
    bf.bf_bank_destroy(bank)


@pytest.mark.parametrize("case", ["dc_offset", "spike"])
def test_offset_and_spike(ctx, case):
    """A large DC offset (partial sums of the offset times the template's
    running sum) and a single sample 1e5 times the noise (its FFT segments
    send nearly every other lag to the direct fixup; the prefix of x^2 jumps
    by 1e10): dense rho on every route matches the oracle."""
    fs, M = 2048.0, 2048
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC, synth.BOTH], [1.0],
                           40.0, 900.0, 3, 4)                    # 72 templates
    bank = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, STORE_ALL)
    p = oracle_params(spec)
    rng = np.random.default_rng(91)
    x = rng.standard_normal(12500)
    if case == "dc_offset":
        x += 50.0
    else:
        x[6001] = 1e5
    x = x.astype(np.float32)
    ref = oracle.search(x, fs, p, M, want_rho=True)
    K, L = ref["rho"].shape
    for prec in ("split_bf16", "fp32", "split_fp16", "fft_fp32", "bf16"):
        rho = torch.zeros((K, L), dtype=torch.float32, device="cuda")
        outs, _, _ = run(ctx, bank, [x], fs, prec, rho_out=rho)
        err = np.abs(rho.cpu().numpy().astype(np.float64) - ref["rho"])
        assert err.max() <= TOL[prec], (prec, err.max(), np.unravel_index(err.argmax(), err.shape))
        check_maxima(outs[0], ref, ref["rho"], TOL[prec], prec)
    bf.bf_bank_destroy(bank)
