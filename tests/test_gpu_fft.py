"""GPU parity of the FFT route (BF_FFT_FP32: overlap-save over segments of
16384 samples with plain banks, 8192 with quadrature banks; template spectra
kept with the bank) against the oracle, at sizes that span several segments
with a ragged last one, and at the full GW size on sampled templates."""
import numpy as np
import pytest

import oracle
from paper_1802_01685_gb300 import bf, synth

from parity import TOL, check_hist, check_maxima, check_sigma, oracle_params, run, subset

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PREC = "fft_fp32"
F = 16384                    # samples per segment with a plain bank


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = bf.bf_init()
    yield h
    bf.bf_destroy(h)


def test_gw_cut_down_several_segments(ctx):
    """M = 4096: 12,289 lags per segment, 28,673 lags = three segments, the
    last one 4,095 lags.  Dense rho across the seams, maxima, sigma and
    histogram of the data and both controls."""
    w = synth.gw_pair(n=32768, I=16, J=16)
    fs, M = w["fs"], w["M"]
    xs = w["series"]
    ctrl = [bf.bf_control_randomize(ctx, x, sd) for x, sd in zip(xs, w["control_seeds"])]
    p = oracle_params(w["grid"])
    refs = [oracle.search(x, fs, p, M, want_rho=True) for x in xs + ctrl]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_SPLIT_BF16)
    K, L = refs[0]["rho"].shape
    assert L == 28673 and -(-L // (F - M + 1)) == 3
    rho = torch.zeros((K, L), dtype=torch.float32, device="cuda")
    run(ctx, bank, xs[:1], fs, PREC, rho_out=rho)
    err = np.abs(rho.cpu().numpy().astype(np.float64) - refs[0]["rho"])
    assert err.max() <= TOL[PREC], err.max()
    # the lags on either side of each seam
    for t in (12287, 12288, 12289, 24577, 24578, L - 1):
        assert err[:, t].max() <= TOL[PREC]
    outs, mean, info = run(ctx, bank, xs + ctrl, fs, PREC)
    assert info.correlations == 4 * K * L and info.tile_lags == 0
    for s, (g, r) in enumerate(zip(outs, refs)):
        check_maxima(g, r, r["rho"], TOL[PREC], f"series {s}")
        check_sigma(g, r, TOL[PREC])
        check_hist(g["hist"], r["max"], TOL[PREC])
    bf.bf_bank_destroy(bank)


def test_grb_cut_down_uneven_batch(ctx):
    """M = 2000 (6193 lags per segment), four light curves of 10-20 s in one
    launch, both senses, mean spectrum over the batch."""
    w = synth.grb_batch(n_series=4, t_min=10.0, t_max=20.0, I=8, J=8)
    fs, M = w["fs"], w["M"]
    xs = w["series"]
    p = oracle_params(w["grid"])
    refs = [oracle.search(x, fs, p, M, want_rho=True) for x in xs]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0)
    outs, mean, _ = run(ctx, bank, xs, fs, PREC)
    for s, (g, r) in enumerate(zip(outs, refs)):
        check_maxima(g, r, r["rho"], TOL[PREC], f"series {s}")
        check_sigma(g, r, TOL[PREC])
    np.testing.assert_allclose(mean, np.mean([r["max"] for r in refs], axis=0), atol=TOL[PREC])
    bf.bf_bank_destroy(bank)


def test_odd_bank_slice_and_generated_bank(ctx):
    """An odd number of templates (the last one has no partner in its
    transform), starting at an odd index; the same from a bank that stores
    only the chirp parameters."""
    w = synth.tiny(seed=3)
    fs, M = w["fs"], w["M"]
    x = w["series"][0]
    p = oracle_params(w["grid"])
    b0, b1 = 3, 200
    ref = oracle.search(x, fs, subset(p, np.arange(b0, b1)), M, want_rho=True)
    for storage in (bf.BF_BANK_FP32, bf.BF_BANK_GENERATED):
        bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, storage)
        outs, _, info = run(ctx, bank, [x], fs, PREC, bank_begin=b0, bank_end=b1)
        assert info.n_templates == b1 - b0
        check_maxima(outs[0], ref, ref["rho"], TOL[PREC], f"storage {storage}")
        check_sigma(outs[0], ref, TOL[PREC])
        bf.bf_bank_destroy(bank)


def test_agrees_with_the_direct_path(ctx):
    """The FFT route and the split-BF16 tensor-core path on the same ragged
    batch: maxima within the sum of their tolerances; tails the same set up
    to values within that bound of the threshold."""
    fs, M = 4096.0, 4096
    spec = synth.grid_spec([synth.POWERLAW, synth.LINEAR], [synth.ASC, synth.DESC], [1.0, 0.6],
                           30.0, 900.0, 6, 6)                    # 288 templates
    bank = bf.bf_bank_create_grid(ctx, spec, fs, 1.0)
    rng = np.random.default_rng(77)
    xs = [synth.gw_coloured(n, fs, rng).astype(np.float32) for n in (M, 9000, 30001, 50000)]
    kappa = 4.0
    a = run(ctx, bank, xs, fs, PREC, want_tails=True, kappa=kappa)[0]
    b = run(ctx, bank, xs, fs, "split_bf16", want_tails=True, kappa=kappa)[0]
    for ga, gb in zip(a, b):
        assert np.abs(ga["max"].astype(np.float64) - gb["max"]).max() <= 2 * TOL[PREC]
        assert np.abs(ga["sigma"].astype(np.float64) - gb["sigma"]).max() <= 2 * TOL[PREC]
    bf.bf_bank_destroy(bank)


def test_full_size_gw_pair_sampled(ctx):
    """Both 64 s series against all 65,536 templates (21 segments each);
    twelve templates spread over the bank recomputed by the oracle over every
    lag of series 0; the whole output against the split-BF16 path."""
    w = synth.gw_pair()
    fs, M = w["fs"], w["M"]
    xs = w["series"]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_SPLIT_BF16)
    outs, mean, info = run(ctx, bank, xs, fs, PREC)
    assert info.correlations == 2 * (len(xs[0]) - M + 1) * 65536
    p = oracle_params(w["grid"])
    idx = np.array([0, 1, 255, 4096, 20000, 32767, 32768, 40000, 50000, 60001, 65534, 65535])
    ref = oracle.search(xs[0], fs, subset(p, idx), M, want_rho=True)
    g = {k: v[idx] for k, v in outs[0].items() if k in ("max", "argmax", "sigma")}
    check_maxima(g, ref, ref["rho"], TOL[PREC], "full size")
    check_sigma(g, ref, TOL[PREC])
    direct = run(ctx, bank, xs, fs, "split_bf16")[0]
    for ga, gb in zip(outs, direct):
        assert np.abs(ga["max"].astype(np.float64) - gb["max"]).max() <= 2 * TOL[PREC]
        assert ga["hist"].sum() == 65536
    bf.bf_bank_destroy(bank)


def test_rejections(ctx):
    """Templates longer than half a transform answer BF_ENOTSUP."""
    fs = 8192.0
    bank = bf.bf_bank_create(ctx, [(bf.BF_LINEAR, bf.BF_ASC, 100.0, 2000.0, 1.0)], fs, 1.0)
    x = np.random.default_rng(1).standard_normal(20000).astype(np.float32)
    with pytest.raises(bf.BFError) as e:
        run(ctx, bank, [x], fs, PREC)
    assert e.value.status == bf.BF_ENOTSUP
    bf.bf_bank_destroy(bank)


def test_generated_bank_in_chunks(ctx):
    """A bank that keeps only chirp parameters makes its spectra 8,192 rows
    at a time in a two-slot ring: a 20,000-template bank from an odd offset
    spans three chunks.  Templates around the chunk edges against the oracle;
    every template against the bank that keeps its spectra."""
    fs, M = 2048.0, 2048
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0], 20.0,
                           1000.0, 50, 100)                      # 20,000 templates
    x = np.random.default_rng(23).standard_normal(12000).astype(np.float32)
    b0 = 7
    gen = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, bf.BF_BANK_GENERATED)
    outs, _, info = run(ctx, gen, [x], fs, PREC, bank_begin=b0)
    g = outs[0]
    assert info.n_templates == 20000 - b0
    p = oracle_params(spec)
    idx = np.array([0, 1, 8190, 8191, 8192, 8193, 16382, 16383, 16384, 16385, 19991, 19992])
    idx = idx[idx < 20000 - b0]
    ref = oracle.search(x, fs, subset(p, idx + b0), M, want_rho=True)
    gs = {k: v[idx] for k, v in g.items() if k in ("max", "argmax", "sigma")}
    check_maxima(gs, ref, ref["rho"], TOL[PREC], "chunk edge")
    check_sigma(gs, ref, TOL[PREC])
    stored = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, bf.BF_BANK_FP32)
    s = run(ctx, stored, [x], fs, PREC, bank_begin=b0)[0][0]
    assert np.abs(s["max"].astype(np.float64) - g["max"]).max() <= 2 * TOL[PREC]
    assert np.abs(s["sigma"].astype(np.float64) - g["sigma"]).max() <= 2 * TOL[PREC]
    bf.bf_bank_destroy(stored)
    bf.bf_bank_destroy(gen)


def test_plan_on_generated_bank_in_chunks(ctx):
    """A plan on a 20,000-template generated bank captures the spectra ring
    (three chunks of 8,192 rows made on the auxiliary stream) in its graph:
    replays equal bf_correlate on the same bank bit for bit, and the oracle
    around the chunk edges."""
    fs, M = 2048.0, 2048
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0], 20.0,
                           1000.0, 50, 100)                      # 20,000 templates
    gen = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, bf.BF_BANK_GENERATED)
    p = oracle_params(spec)
    b0 = 7
    idx = np.array([0, 8191, 8192, 16383, 16384, 19992])
    opts = bf.make_opts(precision=PREC, bank_begin=b0, want_tails=True, kappa=4.0)
    lens = [12000, 3000]
    plan = bf.bf_plan_create(ctx, gen, lens, fs, opts)
    try:
        for run_i in range(2):
            rng = np.random.default_rng(230 + run_i)
            xs = [rng.standard_normal(n).astype(np.float32) for n in lens]
            res = bf.bf_plan_run(plan, xs)
            got = [bf.bf_result_copy_to_host(res, s) for s in range(len(lens))]
            got_t = np.sort(bf.bf_result_copy_tails(res), order=["series", "k", "tau"])
            ref_h = bf.bf_correlate(ctx, gen, xs, fs, opts)
            ref = [bf.bf_result_copy_to_host(ref_h, s) for s in range(len(lens))]
            ref_t = np.sort(bf.bf_result_copy_tails(ref_h), order=["series", "k", "tau"])
            bf.bf_result_destroy(ref_h)
            for g, r in zip(got, ref):
                np.testing.assert_array_equal(g["max"], r["max"])
                np.testing.assert_array_equal(g["argmax"], r["argmax"])
                np.testing.assert_array_equal(g["hist"], r["hist"])
            np.testing.assert_array_equal(got_t, ref_t)
            o = oracle.search(xs[0], fs, subset(p, idx + b0), M, want_rho=True)
            gs = {k: v[idx] for k, v in got[0].items() if k in ("max", "argmax", "sigma")}
            check_maxima(gs, o, o["rho"], TOL[PREC], "plan, chunk edges")
    finally:
        bf.bf_plan_destroy(plan)
    bf.bf_bank_destroy(gen)


def test_spectra_over_the_budget():
    """Template spectra that do not fit the context's HBM budget give
    BF_ENOMEM and leave the context usable; a generated bank needs only its
    ring and goes through."""
    import __graft_entry__
    __graft_entry__.build()
    cfg = bf.bf_config_default()
    cfg.hbm_budget = 256 << 20                      # 256 MiB
    ctx = bf.bf_init(cfg)
    try:
        fs, M = 2048.0, 2048
        spec = synth.grid_spec([synth.LINEAR], [synth.ASC, synth.DESC], [1.0], 20.0, 1000.0, 64, 64)
        x = np.random.default_rng(31).standard_normal(10000).astype(np.float32)
        stored = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, bf.BF_BANK_FP32)   # 8192 x 2048 floats
        with pytest.raises(bf.BFError) as e:                # 8192 x 64 KiB of spectra
            run(ctx, stored, [x], fs, PREC)
        assert e.value.status == bf.BF_ENOMEM
        a = run(ctx, stored, [x], fs, "fp32", bank_end=512)[0][0]
        bf.bf_bank_destroy(stored)
        gen = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, bf.BF_BANK_GENERATED)
        b = run(ctx, gen, [x], fs, PREC, bank_end=512)[0][0]
        assert np.abs(a["max"].astype(np.float64) - b["max"]).max() <= 2 * TOL[PREC]
        bf.bf_bank_destroy(gen)
    finally:
        bf.bf_destroy(ctx)


@pytest.mark.parametrize("fs,T", [(64.0, 1.0), (2.0, 1.0), (1000.0, 1.0), (4096.0, 1.0)])
def test_template_lengths(ctx, fs, T):
    """Template lengths from 2 to 4096 samples (up to 16383 lags per
    segment), series of one segment, of several and of exactly one lag."""
    M = int(round(T * fs))
    ny = fs / 2
    chirps = [(bf.BF_LINEAR, bf.BF_ASC, 0.1 * ny, 0.8 * ny, 1.0 * T),
              (bf.BF_POWERLAW, bf.BF_DESC, 0.05 * ny, 0.6 * ny, 0.7 * T),
              (bf.BF_LINEAR, bf.BF_BOTH, 0.2 * ny, 0.5 * ny, 0.9 * T)]
    if M < 8:
        chirps = chirps[:1]
    bank = bf.bf_bank_create(ctx, chirps, fs, T)
    p = dict(track=np.array([c[0] for c in chirps], np.int32), sense=np.array([c[1] for c in chirps], np.int32),
             f_lo=np.array([c[2] for c in chirps]), f_hi=np.array([c[3] for c in chirps]),
             D=np.array([c[4] for c in chirps]))
    rng = np.random.default_rng(M)
    for n in (M, M + 5, 3 * F + 17):
        x = rng.standard_normal(n).astype(np.float32)
        ref = oracle.search(x, fs, p, M, want_rho=True)
        K, L = ref["rho"].shape
        rho = torch.zeros((K, L), dtype=torch.float32, device="cuda")
        outs, _, _ = run(ctx, bank, [x], fs, PREC, rho_out=rho)
        assert np.abs(rho.cpu().numpy() - ref["rho"]).max() <= TOL[PREC], (M, n)
        check_maxima(outs[0], ref, ref["rho"], TOL[PREC], f"M={M} n={n}")
    bf.bf_bank_destroy(bank)


def _quiet_loud_series(rng, n, quiet, scale):
    """White noise with the stretches in `quiet` scaled by `scale`."""
    x = rng.standard_normal(n)
    for a, b in quiet:
        x[a:b] *= scale
    return x


@pytest.mark.parametrize("quad", [False, True])
def test_low_energy_windows_computed_directly(ctx, quad):
    """Windows that hold almost none of their segment's energy: the tapered
    edges of a chirp alone in silence, and a stretch of noise 10^5 times
    quieter than its neighbours.  The transform's rounding error scales with
    the segment, so these lags go to the direct fixup; dense rho, maxima,
    sigma, tails and map all match the oracle, and rho never exceeds 1."""
    fs, M = 2048.0, 2048
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC, synth.BOTH],
                           [1.0, 0.5], 40.0, 900.0, 3, 5)        # 180 chirps
    p = oracle_params(spec)
    rng = np.random.default_rng(71)
    storage = bf.BF_BANK_SPLIT_BF16 | (bf.BF_BANK_QUADRATURE if quad else 0)
    bank = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, storage)
    # series 0: zeros with a bank template placed at 5000, 3 times its size
    x0 = np.zeros(14000)
    x0[5000:5000 + M] = 3.0 * oracle.template(int(p["track"][17]), int(p["sense"][17]), p["f_lo"][17],
                                              p["f_hi"][17], p["D"][17], fs, M, 0)
    # series 1: noise with a stretch 1e-5 as loud (windows inside it are
    # normalised noise again, as loud in rho as the rest)
    x1 = _quiet_loud_series(rng, 16000, [(6000, 11000)], 1e-5)
    xs = [x0.astype(np.float32), x1.astype(np.float32)]
    kappa = 2.5 if quad else 4.0       # phase-blind output: |rho|^2 M / 2 is chi^2 with 2 dof on noise
    tol = TOL[PREC]
    for s, x in enumerate(xs):
        ref = oracle.search(x, fs, p, M, want_rho=True, quadrature=quad)
        K, L = ref["rho"].shape
        rho = torch.zeros((K, L), dtype=torch.float32, device="cuda")
        outs, _, _ = run(ctx, bank, [x], fs, PREC, rho_out=rho)
        got = rho.cpu().numpy().astype(np.float64)
        assert np.abs(got).max() <= 1.0 + tol
        err = np.abs(got - ref["rho"])
        assert err.max() <= tol, (s, err.max(), np.unravel_index(err.argmax(), err.shape))
        check_maxima(outs[0], ref, ref["rho"], tol, f"series {s}")
        check_sigma(outs[0], ref, tol)
        if s == 0:
            assert abs(float(outs[0]["max"][17]) - 1.0) <= tol
            if not quad:
                assert outs[0]["argmax"][17] == 5000
        # tails and map against the oracle at the same threshold
        thr = kappa * np.sqrt((2.0 if quad else 1.0) / M)
        res = bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts(precision=PREC, kappa=kappa, want_tails=True,
                                                               want_map=True))
        tails = bf.bf_result_copy_tails(res)
        mp = bf.bf_result_copy_to_host(res, 0, want_map=True)["map"]
        bf.bf_result_destroy(res)
        a = np.abs(ref["rho"])
        got_t = {(int(t["k"]), int(t["tau"])) for t in tails}
        must = set(zip(*[v.tolist() for v in np.nonzero(a >= thr + tol)]))
        may = set(zip(*[v.tolist() for v in np.nonzero(a >= thr - tol)]))
        assert len(must) > 0 and must <= got_t <= may
        hi = oracle.search(x, fs, p, M, thr=thr + tol, want_map=True, quadrature=quad)["map"]
        lo = oracle.search(x, fs, p, M, thr=thr - tol, want_map=True, quadrature=quad)["map"]
        assert np.all(mp >= hi - tol) and np.all(mp <= lo + tol)
    bf.bf_bank_destroy(bank)


def test_low_energy_windows_in_plans_generated_banks_and_serving(ctx):
    """The fixup runs inside a captured plan, with a generated bank (spectra
    made chunk by chunk) and in the serving loop, giving what bf_correlate
    gives with a stored bank."""
    fs, M = 2048.0, 2048
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0], 40.0, 900.0, 4, 8)
    rng = np.random.default_rng(72)
    xs = [_quiet_loud_series(rng, n, [(3000, 7000)], 1e-6).astype(np.float32) for n in (12000, 9000)]
    stored = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, bf.BF_BANK_SPLIT_BF16)
    gen = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, bf.BF_BANK_GENERATED)
    opts = bf.make_opts(precision=PREC, want_tails=True)

    def outputs(res, owned=True):
        o = [bf.bf_result_copy_to_host(res, s) for s in range(len(xs))]
        t = np.sort(bf.bf_result_copy_tails(res), order=["series", "k", "tau"])
        if owned:
            bf.bf_result_destroy(res)
        return o, t

    ref, ref_t = outputs(bf.bf_correlate(ctx, stored, xs, fs, opts))
    p = oracle_params(spec)
    for s, x in enumerate(xs):
        r = oracle.search(x, fs, p, M, want_rho=True)
        check_maxima(ref[s], r, r["rho"], TOL[PREC], f"series {s}")
    g, g_t = outputs(bf.bf_correlate(ctx, gen, xs, fs, opts))
    plan = bf.bf_plan_create(ctx, stored, [len(x) for x in xs], fs, opts)
    try:
        for _ in range(2):
            pl, pl_t = outputs(bf.bf_plan_run(plan, xs), owned=False)     # the plan's result
            for a, b in zip(ref, pl):
                np.testing.assert_array_equal(a["max"], b["max"])
                np.testing.assert_array_equal(a["argmax"], b["argmax"])
            np.testing.assert_array_equal(ref_t, pl_t)
    finally:
        bf.bf_plan_destroy(plan)
    for a, b in zip(ref, g):
        np.testing.assert_array_equal(a["max"], b["max"])
        np.testing.assert_array_equal(a["argmax"], b["argmax"])
    np.testing.assert_array_equal(ref_t, g_t)
    for s, x in enumerate(xs):
        t = bf.bf_serve_submit(ctx, stored, x, fs, opts)
        st, res = bf.bf_serve_poll(ctx, t, 60_000_000)
        assert st == bf.BF_OK
        srv = bf.bf_result_copy_to_host(res, 0)
        bf.bf_result_destroy(res)
        np.testing.assert_array_equal(srv["max"], ref[s]["max"])
        np.testing.assert_array_equal(srv["argmax"], ref[s]["argmax"])
    bf.bf_bank_destroy(stored)
    bf.bf_bank_destroy(gen)
