"""GPU parity of quadrature banks (BF_BANK_QUADRATURE: every chirp with its
Hilbert partner, output sqrt(rho_cos^2 + rho_sin^2)) against the oracle, on
every correlation route."""
import numpy as np
import pytest

import oracle
from paper_1802_01685_gb300 import bf, synth

from parity import (STORE_ALL, TOL, check_maxima, check_sigma, check_template_rows, oracle_params, run,
                    subset)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PRECS = ["split_bf16", "fp32", "bf16", "fft_fp32", "split_fp16"]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = bf.bf_init()
    yield h
    bf.bf_destroy(h)


@pytest.fixture(scope="module")
def case(ctx):
    """Both tracks and senses and the superposition; a chirp injected with
    an arbitrary phase (a mix of its template and partner) into white noise;
    a ragged number of lags; 2 x 2 x 3 x 4 x 4 + 32 = 224 chirps (448 rows,
    more than three template tiles)."""
    fs, M = 2048.0, 2048
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC, synth.BOTH],
                           [1.0, 0.6], 40.0, 900.0, 4, 4)       # 192 chirps
    p = oracle_params(spec)
    extra = synth.grid_spec([synth.LINEAR], [synth.DESC], [0.8], 100.0, 700.0, 4, 8)
    pe = oracle_params(extra)
    p = {k: np.concatenate([p[k], pe[k]]) for k in p}
    K = len(p["track"])
    chirps = [(int(p["track"][k]), int(p["sense"][k]), float(p["f_lo"][k]), float(p["f_hi"][k]),
               float(p["D"][k])) for k in range(K)]
    rng = np.random.default_rng(61)
    x = rng.standard_normal(9300)
    k_inj, n0, phi = 77, 3111, 1.1
    hc = oracle.template(*chirps[k_inj], fs, M, 0)
    hs = oracle.template(*chirps[k_inj], fs, M, 1)
    x[n0:n0 + M] += 12.0 * (np.cos(phi) * hc + np.sin(phi) * hs)
    x = x.astype(np.float32)
    ref = oracle.search(x, fs, p, M, want_rho=True, quadrature=True)
    return dict(fs=fs, M=M, p=p, chirps=chirps, x=x, ref=ref, k_inj=k_inj, n0=n0)


def test_bank_rows_are_the_pairs(ctx, case):
    """Stored and generated quadrature banks hold template and partner as
    rows 2k, 2k + 1: the FP32 rows within 2e-6 (L2) of the oracle's pairs,
    the split layouts the exact splits of those rows, and the generated bank
    the stored one bit for bit."""
    fs, M, chirps = case["fs"], case["M"], case["chirps"]
    idx = [0, 5, 77, 150, 223]
    ref = np.stack([oracle.template(*chirps[k], fs, M, ph) for k in idx for ph in (0, 1)])
    rows = {}
    for name, storage in (("f32", bf.BF_BANK_FP32), ("bf16", bf.BF_BANK_SPLIT_BF16),
                          ("fp16", bf.BF_BANK_SPLIT_FP16), ("gen", bf.BF_BANK_GENERATED)):
        bank = bf.bf_bank_create(ctx, chirps, fs, 1.0, storage | bf.BF_BANK_QUADRATURE)
        assert bf.bf_bank_size(bank) == len(chirps) and bf.bf_bank_rows(bank) == 2 * len(chirps)
        rows[name] = np.concatenate([bf.bf_bank_read(bank, k, 1) for k in idx])
        assert rows[name].shape == (2 * len(idx), M)
        bf.bf_bank_destroy(bank)
    np.testing.assert_array_equal(rows["gen"], rows["f32"])
    check_template_rows(rows["f32"], {"bf16": rows["bf16"], "fp16": rows["fp16"]}, ref)


@pytest.mark.parametrize("prec", PRECS)
def test_dense_output_maxima_sigma(ctx, case, prec):
    fs, M, x, ref = case["fs"], case["M"], case["x"], case["ref"]
    storage = STORE_ALL | bf.BF_BANK_QUADRATURE
    bank = bf.bf_bank_create(ctx, case["chirps"], fs, 1.0, storage)
    K, L = ref["rho"].shape
    rho = torch.zeros((K, L), dtype=torch.float32, device="cuda")
    outs, _, info = run(ctx, bank, [x], fs, prec, rho_out=rho)
    assert info.n_templates == K and info.correlations == 2 * K * L
    err = np.abs(rho.cpu().numpy().astype(np.float64) - ref["rho"])
    assert err.max() <= TOL[prec], err.max()
    check_maxima(outs[0], ref, ref["rho"], TOL[prec], prec)
    check_sigma(outs[0], ref, TOL[prec])
    # the phase-blind output follows the envelope, whose top is flat to a lag or two
    assert abs(int(outs[0]["argmax"][case["k_inj"]]) - case["n0"]) <= 2
    assert abs(int(ref["argmax"][case["k_inj"]]) - case["n0"]) <= 2
    # without the dense output (the fused path that the benchmark times)
    g = run(ctx, bank, [x], fs, prec)[0][0]
    check_maxima(g, ref, ref["rho"], TOL[prec], prec)
    bf.bf_bank_destroy(bank)


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "fft_fp32", "split_fp16"])
def test_tails_map_and_slice(ctx, case, prec):
    """Tails |rho_q| >= kappa sqrt(2/M) and the map they paint, on an odd
    slice of the bank (a partial template tile at both ends)."""
    fs, M, x, p = case["fs"], case["M"], case["x"], case["p"]
    b0, b1 = 13, 201
    ps = subset(p, np.arange(b0, b1))
    kappa, tol = 4.0, TOL[prec]
    thr = kappa * np.sqrt(2.0 / M)
    ref = oracle.search(x, fs, ps, M, want_rho=True, quadrature=True, thr=thr)
    bank = bf.bf_bank_create(ctx, case["chirps"], fs, 1.0, STORE_ALL | bf.BF_BANK_QUADRATURE)
    res = bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts(precision=prec, bank_begin=b0, bank_end=b1,
                                                           kappa=kappa, want_tails=True, want_map=True))
    info = bf.bf_result_info_get(res)
    assert abs(info.threshold - thr) < 1e-7
    tails = bf.bf_result_copy_tails(res)
    g = bf.bf_result_copy_to_host(res, 0, want_map=True)
    bf.bf_result_destroy(res)
    check_maxima(g, ref, ref["rho"], tol, prec)
    a = ref["rho"]
    got = {(int(t["k"]) - b0, int(t["tau"])): float(t["rho"]) for t in tails}
    must = set(zip(*[v.tolist() for v in np.nonzero(a >= thr + tol)]))
    may = set(zip(*[v.tolist() for v in np.nonzero(a >= thr - tol)]))
    assert len(must) > 0 and must <= set(got) <= may
    for (k, tau), r in got.items():
        assert abs(r - a[k, tau]) <= tol and r >= 0
    hi = oracle.search(x, fs, ps, M, thr=thr + tol, want_map=True, quadrature=True)["map"]
    lo = oracle.search(x, fs, ps, M, thr=thr - tol, want_map=True, quadrature=True)["map"]
    assert np.all(g["map"] >= hi - tol) and np.all(g["map"] <= lo + tol)
    bf.bf_bank_destroy(bank)


def test_generated_bank_equals_stored(ctx, case):
    fs, x = case["fs"], case["x"]
    stored = bf.bf_bank_create(ctx, case["chirps"], fs, 1.0, bf.BF_BANK_SPLIT_BF16 | bf.BF_BANK_QUADRATURE)
    gen = bf.bf_bank_create(ctx, case["chirps"], fs, 1.0, bf.BF_BANK_GENERATED | bf.BF_BANK_QUADRATURE)
    for prec in ("split_bf16", "fp32", "split_fp16"):
        if prec != "split_bf16":
            bf.bf_bank_destroy(stored)
            layout = bf.BF_BANK_FP32 if prec == "fp32" else bf.BF_BANK_SPLIT_FP16
            stored = bf.bf_bank_create(ctx, case["chirps"], fs, 1.0, layout | bf.BF_BANK_QUADRATURE)
        a = run(ctx, stored, [x], fs, prec, bank_begin=9, bank_end=220)[0][0]
        b = run(ctx, gen, [x], fs, prec, bank_begin=9, bank_end=220)[0][0]
        np.testing.assert_array_equal(a["max"], b["max"])
        np.testing.assert_array_equal(a["argmax"], b["argmax"])
    bf.bf_bank_destroy(stored)
    bf.bf_bank_destroy(gen)


def test_parseval_sigma_of_pairs(ctx, case):
    """The predicted sigma of a quadrature output is the root of the summed
    squares of the pair's predictions."""
    fs, M, x, p = case["fs"], case["M"], case["x"], case["p"]
    bank = bf.bf_bank_create(ctx, case["chirps"], fs, 1.0, bf.BF_BANK_SPLIT_BF16 | bf.BF_BANK_QUADRATURE)
    res = bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts(tail_sigma=bf.BF_SIGMA_PARSEVAL, bank_begin=3,
                                                           bank_end=100))
    got = bf.bf_result_copy_sigma_pred(res, 0)
    bf.bf_result_destroy(res)
    sub = subset(p, np.arange(3, 100))
    sc = oracle.parseval_sigma(x, oracle.bank(sub, fs, M, 0))
    ss = oracle.parseval_sigma(x, oracle.bank(sub, fs, M, 1))
    np.testing.assert_allclose(got, np.sqrt(sc ** 2 + ss ** 2), rtol=2e-5)
    bf.bf_bank_destroy(bank)
