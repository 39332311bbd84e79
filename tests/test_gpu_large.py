"""GPU parity on the paper-shaped workloads: cut-down versions checked in
full against the oracle, and the full-size GW pair checked on sampled
templates."""
import numpy as np
import pytest

import oracle
from paper_1802_01685_gb300 import bf, synth

from parity import TOL, check_hist, check_map, check_maxima, check_sigma, oracle_params, run, subset

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = bf.bf_init()
    yield h
    bf.bf_destroy(h)


def test_gw_pair_cut_down_with_controls(ctx):
    """Coloured noise pair with a common power-law chirp and both
    time-randomised controls, all precisions, every template."""
    w = synth.gw_pair(n=16384, I=16, J=16)
    fs, M = w["fs"], w["M"]
    xs = w["series"]
    ctrl = [bf.bf_control_randomize(ctx, x, sd) for x, sd in zip(xs, w["control_seeds"])]
    for c, x, sd in zip(ctrl, xs, w["control_seeds"]):
        np.testing.assert_array_equal(c, oracle.permute(x, sd))
    p = oracle_params(w["grid"])
    refs = [oracle.search(x, fs, p, M, want_rho=True) for x in xs + ctrl]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0)
    for prec in ("split_bf16", "fp32", "bf16"):
        outs, mean, _ = run(ctx, bank, xs + ctrl, fs, prec)
        for s, (g, r) in enumerate(zip(outs, refs)):
            check_maxima(g, r, r["rho"], TOL[prec], f"{prec} series {s}")
            check_sigma(g, r, TOL[prec])
            check_hist(g["hist"], r["max"], TOL[prec])
    # the injected chirp stands out in the data (near its offset), not in the controls
    k = int(np.argmax(refs[0]["max"]))
    assert abs(int(refs[0]["argmax"][k]) - w["n0"][0]) < M // 4
    assert refs[0]["max"].max() > 1.3 * max(refs[2]["max"].max(), refs[3]["max"].max())
    bf.bf_bank_destroy(bank)


def test_gw_pair_full_size_sampled(ctx):
    """Both 64 s series against all 65,536 templates in the launch shape the
    benchmark times; 12 templates spread over the bank recomputed by the
    oracle over every lag of series 0."""
    w = synth.gw_pair()
    fs, M = w["fs"], w["M"]
    xs = w["series"]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_SPLIT_BF16 | bf.BF_BANK_SPLIT_FP16)
    p = oracle_params(w["grid"])
    idx = np.array([0, 1, 255, 4096, 20000, 32767, 32768, 40000, 50000, 60001, 65534, 65535])
    ref = oracle.search(xs[0], fs, subset(p, idx), M, want_rho=True)
    for prec in ("split_bf16", "split_fp16"):
        outs, mean, info = run(ctx, bank, xs, fs, prec)
        assert info.correlations == 2 * (len(xs[0]) - M + 1) * 65536
        g = {k: v[idx] for k, v in outs[0].items() if k in ("max", "argmax", "sigma")}
        check_maxima(g, ref, ref["rho"], TOL[prec], f"full size {prec}")
        check_sigma(g, ref, TOL[prec])
        # properties that hold at any size
        for o in outs:
            assert np.all(o["max"] <= 1.0 + 1e-5) and np.all(o["max"] > 0)
            assert o["hist"].sum() == 65536
            assert np.all(o["argmax"] >= 0) and np.all(o["argmax"] < len(xs[0]) - M + 1)
        np.testing.assert_allclose(mean, (outs[0]["max"].astype(np.float64) + outs[1]["max"]) / 2,
                                   rtol=1e-6)
    bf.bf_bank_destroy(bank)


def test_grb_batch_cut_down(ctx):
    """Poisson light curves at 0.5 ms bins (M = 2000, padded to 2048 inside
    the library), uneven lengths in one launch, both senses, mean spectrum."""
    w = synth.grb_batch(n_series=4, t_min=10.0, t_max=20.0, I=8, J=8)
    fs, M = w["fs"], w["M"]
    xs = w["series"]
    p = oracle_params(w["grid"])
    refs = [oracle.search(x, fs, p, M, want_rho=True) for x in xs]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0)
    assert bf.bf_bank_template_len(bank) == 2000
    for prec in ("split_bf16", "fp32"):
        outs, mean, _ = run(ctx, bank, xs, fs, prec)
        for s, (g, r) in enumerate(zip(outs, refs)):
            check_maxima(g, r, r["rho"], TOL[prec], f"{prec} series {s}")
        ref_mean = np.mean([r["max"] for r in refs], axis=0)
        np.testing.assert_allclose(mean, ref_mean, atol=TOL[prec])
    bf.bf_bank_destroy(bank)


def test_full_bank_grid_cut_down_with_map(ctx):
    """Both tracks, both senses, nine sweep times 0.2..1.0 s; three injected
    chirps; histogram and 1 ms x 4 Hz map."""
    w = synth.full_bank(n=16384, I=3, J=2)
    fs, M = w["fs"], w["M"]
    x = w["series"][0]
    p = oracle_params(w["grid"])
    assert len(p["track"]) == 2 * 2 * 9 * 3 * 2
    ref = oracle.search(x, fs, p, M, want_rho=True)
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0)
    for prec in ("split_bf16", "fp32"):
        outs, _, info = run(ctx, bank, [x], fs, prec, want_map=True)
        g = outs[0]
        check_maxima(g, ref, ref["rho"], TOL[prec], prec)
        check_hist(g["hist"], ref["max"], TOL[prec])
        assert info.candidates_overflow == 0
        check_map(g["map"], x, fs, p, M, 5.0, TOL[prec])
    bf.bf_bank_destroy(bank)


def test_long_templates(ctx):
    """Largest template length used here: 1 s at 16 kHz (M = 16000)."""
    fs = 16000.0
    chirps = [(bf.BF_LINEAR, bf.BF_ASC, 100.0, 7000.0, 1.0), (bf.BF_POWERLAW, bf.BF_DESC, 50.0, 3000.0, 0.7),
              (bf.BF_LINEAR, bf.BF_DESC, 10.0, 20.0, 0.05)]
    x = np.random.default_rng(9).standard_normal(17000).astype(np.float32)
    bank = bf.bf_bank_create(ctx, chirps, fs, 1.0)
    p = dict(track=np.array([c[0] for c in chirps], np.int32), sense=np.array([c[1] for c in chirps], np.int32),
             f_lo=np.array([c[2] for c in chirps]), f_hi=np.array([c[3] for c in chirps]),
             D=np.array([c[4] for c in chirps]))
    ref = oracle.search(x, fs, p, 16000, want_rho=True)
    for prec in ("split_bf16", "fp32", "bf16"):
        K, L = ref["rho"].shape
        rho = torch.zeros((K, L), dtype=torch.float32, device="cuda")
        run(ctx, bank, [x], fs, prec, rho_out=rho)
        err = np.abs(rho.cpu().numpy() - ref["rho"]).max()
        assert err <= TOL[prec], (prec, err)
    bf.bf_bank_destroy(bank)


def test_full_bank_full_size_sampled(ctx):
    """The 8,640,000-template bank at full size (32 s at 2048 Hz), generated on
    the fly, on the tensor-core path and the FFT route (its spectra made in
    chunks); 16 templates spread over the bank recomputed by the oracle; the
    two routes against each other on every template."""
    w = synth.full_bank()
    fs, M = w["fs"], w["M"]
    x = w["series"][0]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_GENERATED)
    K = bf.bf_bank_size(bank)
    assert K == 8640000
    a = run(ctx, bank, [x], fs, "split_bf16", want_hist=True)[0][0]
    b = run(ctx, bank, [x], fs, "fft_fp32", want_hist=True)[0][0]
    p = oracle_params(w["grid"])
    idx = np.linspace(0, K - 1, 16).astype(np.int64)
    ref = oracle.search(x, fs, subset(p, idx), M, want_rho=True)
    for prec, g in (("split_bf16", a), ("fft_fp32", b)):
        gs = {k: v[idx] for k, v in g.items() if k in ("max", "argmax", "sigma")}
        check_maxima(gs, ref, ref["rho"], TOL[prec], f"full bank {prec}")
        check_sigma(gs, ref, TOL[prec])
        assert g["hist"].sum() == K
    assert np.abs(a["max"].astype(np.float64) - b["max"]).max() <= 2 * TOL["split_bf16"]
    bf.bf_bank_destroy(bank)


def test_grb_batch_all_series_sampled(ctx):
    """All 42 light curves at full length (9.3 M samples) in one batched
    launch against a 2048-template slice of the full 2^20 bank; 16 templates
    of the slice recomputed by the oracle on every series; the mean over
    series."""
    w = synth.grb_batch()
    fs, M = w["fs"], w["M"]
    xs = w["series"]
    assert len(xs) == 42
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_SPLIT_BF16)
    assert bf.bf_bank_size(bank) == 2 ** 20
    b0, b1 = 600000, 602048
    outs, mean, info = run(ctx, bank, xs, fs, "split_bf16", bank_begin=b0, bank_end=b1)
    assert info.correlations == sum(len(x) - M + 1 for x in xs) * (b1 - b0)
    p = oracle_params(w["grid"])
    idx = np.linspace(0, b1 - b0 - 1, 16).astype(np.int64)
    sub = subset(p, idx + b0)
    ref_max = []
    for s, (g, x) in enumerate(zip(outs, xs)):
        r = oracle.search(x, fs, sub, M, want_rho=True)      # one series at a time
        gs = {k: v[idx] for k, v in g.items() if k in ("max", "argmax", "sigma")}
        check_maxima(gs, r, r["rho"], TOL["split_bf16"], f"series {s}")
        ref_max.append(r["max"])
    np.testing.assert_allclose(mean[idx], np.mean(ref_max, axis=0), atol=TOL["split_bf16"])
    bf.bf_bank_destroy(bank)
