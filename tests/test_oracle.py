"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks one definition of the oracle against a library routine, a
closed form, an invariant, brute force on a tiny case, or a published value,
so that a dropped term, a wrong sign or index, or a transposed operand in
``oracle/oracle.c`` fails here.  No GPU is needed.
"""
import json
import os

import numpy as np
import pytest
import scipy.signal
import scipy.stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed):
    return np.random.default_rng(seed)


# ----------------------------------------------------------------- numerator

def test_numerator_and_energy_match_numpy():
    x = rng(11).standard_normal(3000).astype(np.float32)
    h = oracle.template(oracle.LINEAR, oracle.ASC, 80.0, 300.0, 0.25, 1024.0, 512)
    num, en = oracle.correlate_raw(x, h)
    x64 = x.astype(np.float64)
    ref_num = np.correlate(x64, h, mode="valid")
    ref_en = np.convolve(x64 * x64, np.ones(len(h)), mode="valid")
    assert num.shape == (len(x) - len(h) + 1,)
    np.testing.assert_allclose(num, ref_num, rtol=0, atol=1e-11)
    np.testing.assert_allclose(en, ref_en, rtol=1e-13, atol=0)


def test_numerator_brute_force_tiny():
    r = rng(12)
    x = r.standard_normal(40).astype(np.float32)
    h = r.standard_normal(9)
    num, en = oracle.correlate_raw(x, h)
    for tau in range(40 - 9 + 1):
        s = 0.0
        e = 0.0
        for m in range(9):
            s += float(x[tau + m]) * float(h[m])
            e += float(x[tau + m]) ** 2
        assert abs(num[tau] - s) < 1e-13
        assert abs(en[tau] - e) < 1e-13


# ----------------------------------------------------------------- rho closed forms

FS, M = 1024.0, 256


def small_bank():
    return oracle.grid([oracle.LINEAR, oracle.POWERLAW], [oracle.ASC, oracle.DESC],
                       [0.25, 0.15], 20.0, 500.0, 2, 2)


def test_injected_template_recovered_with_rho_one():
    p = small_bank()
    K = len(p["track"])
    N = 5 * M
    for k in [0, 3, K // 2, K - 1]:
        h = oracle.template(int(p["track"][k]), int(p["sense"][k]), p["f_lo"][k],
                            p["f_hi"][k], p["D"][k], FS, M)
        for amp, n0 in [(7.5, 300), (-2.0, 0), (0.125, N - M)]:
            x = np.zeros(N, np.float64)
            x[n0:n0 + M] = amp * h
            x = x.astype(np.float32)
            one = {key: p[key][k:k + 1] for key in p}
            out = oracle.search(x, FS, one, M, want_rho=True)
            # float32 rounding of the injected samples limits exactness
            assert abs(out["rho"][0, n0] - np.sign(amp)) < 1e-6
            assert out["argmax"][0] == n0
            assert abs(out["max"][0] - 1.0) < 1e-6


def test_exact_unit_correlation_with_float_template():
    # template rounded to float32 first, then used as the data: rho = 1 to FP64
    # rounding, because the data window equals the template direction up to the
    # float32 rounding of h, which the test removes by building x from float32.
    h = oracle.template(oracle.LINEAR, oracle.ASC, 100.0, 400.0, 0.2, FS, M)
    x = np.zeros(3 * M, np.float32)
    x[M:2 * M] = h.astype(np.float32)
    num, en = oracle.correlate_raw(x, x[M:2 * M].astype(np.float64))
    assert abs(num[M] / np.sqrt(en[M]) - np.sqrt(en[M])) < 1e-15


def test_zero_window_gives_zero():
    p = small_bank()
    x = np.zeros(4 * M, np.float32)
    x[2 * M + 10:] = rng(3).standard_normal(4 * M - 2 * M - 10)
    out = oracle.search(x, FS, p, M, want_rho=True)
    # windows 0..M+10 are all-zero
    assert np.all(out["rho"][:, :M + 11] == 0.0)
    # once a window holds data, rho is num / sqrt(energy) again
    h = oracle.template(int(p["track"][0]), int(p["sense"][0]), p["f_lo"][0],
                        p["f_hi"][0], p["D"][0], FS, M)
    num, en = oracle.correlate_raw(x, h)
    assert np.all(en[M + 11:] > 0) and np.all(en[:M + 11] == 0)
    np.testing.assert_allclose(out["rho"][0, M + 11:], num[M + 11:] / np.sqrt(en[M + 11:]),
                               rtol=0, atol=1e-15)


def test_cauchy_schwarz_bound():
    p = small_bank()
    x = rng(4).standard_normal(6 * M).astype(np.float32)
    out = oracle.search(x, FS, p, M, want_rho=True)
    assert np.all(np.abs(out["rho"]) <= 1.0 + 1e-12)
    assert np.all(out["max"] <= 1.0 + 1e-12)


def test_scale_invariance():
    p = small_bank()
    x = rng(5).standard_normal(4 * M).astype(np.float32)
    base = oracle.search(x, FS, p, M, want_rho=True)["rho"]
    for a in [-4.0, 0.5, 2.0 ** -10]:
        r = oracle.search((a * x).astype(np.float32), FS, p, M, want_rho=True)["rho"]
        np.testing.assert_allclose(r, np.sign(a) * base, rtol=0, atol=1e-13)
    r = oracle.search((-3.0 * x).astype(np.float32), FS, p, M, want_rho=True)["rho"]
    np.testing.assert_allclose(r, -base, rtol=0, atol=2e-7)


def test_time_shift_invariance():
    p = small_bank()
    x = rng(6).standard_normal(4 * M).astype(np.float32)
    s = 37
    xs = np.concatenate([rng(7).standard_normal(s).astype(np.float32), x])
    a = oracle.search(x, FS, p, M, want_rho=True)["rho"]
    b = oracle.search(xs, FS, p, M, want_rho=True)["rho"]
    np.testing.assert_array_equal(b[:, s:], a)


def test_linearity_of_numerator():
    r = rng(8)
    x1 = r.standard_normal(900).astype(np.float32)
    x2 = r.standard_normal(900).astype(np.float32)
    h = oracle.template(oracle.POWERLAW, oracle.DESC, 60.0, 300.0, 0.2, FS, M)
    n1, _ = oracle.correlate_raw(x1, h)
    n2, _ = oracle.correlate_raw(x2, h)
    n12, _ = oracle.correlate_raw((x1.astype(np.float64) + x2).astype(np.float32), h)
    # x1 + x2 is rounded to float32 once: error bounded by ulp * ||h||_1 terms
    assert np.max(np.abs(n12 - (n1 + n2))) < 1e-5


def test_white_noise_rho_is_beta_distributed():
    """For iid Gaussian x, x/|x| is uniform on the sphere, so (rho+1)/2 is
    Beta((M-1)/2, (M-1)/2) exactly and E[rho^2] = 1/M."""
    Mw = 128
    p = oracle.grid([oracle.LINEAR], [oracle.ASC], [0.1], 30.0, 400.0, 1, 2)
    x = rng(9).standard_normal(Mw * 3000).astype(np.float32)
    out = oracle.search(x, 1024.0, p, Mw, want_rho=True)
    for k in range(2):
        r = out["rho"][k, ::Mw]          # disjoint windows: independent samples
        a = (Mw - 1) / 2.0
        ks = scipy.stats.kstest((r + 1.0) / 2.0, scipy.stats.beta(a, a).cdf)
        assert ks.pvalue > 1e-3, ks
        m2 = np.mean(r * r)
        se = np.sqrt(2.0 / len(r)) / Mw
        assert abs(m2 - 1.0 / Mw) < 5 * se


def test_sigma_is_rms_of_rho_and_argmax_is_first_max():
    p = small_bank()
    x = rng(10).standard_normal(3 * M).astype(np.float32)
    out = oracle.search(x, FS, p, M, want_rho=True)
    rho = out["rho"]
    np.testing.assert_allclose(out["sigma"], np.sqrt(np.mean(rho ** 2, axis=1)), rtol=1e-13)
    a = np.abs(rho)
    np.testing.assert_array_equal(out["max"], a.max(axis=1))
    np.testing.assert_array_equal(out["argmax"], a.argmax(axis=1))  # numpy: first max


def test_argmax_ties_take_smallest_lag():
    # periodic data with period M gives identical windows at lags t and t + M
    h = oracle.template(oracle.LINEAR, oracle.ASC, 100.0, 400.0, 0.2, FS, M)
    one = np.concatenate([h, h, h, h]).astype(np.float32)
    p = oracle.grid([oracle.LINEAR], [oracle.ASC], [0.2], 100.0, 400.0, 1, 1)
    p["f_lo"][:] = 100.0
    p["f_hi"][:] = 400.0
    out = oracle.search(one, FS, p, M, want_rho=True)
    assert out["argmax"][0] == 0
    assert np.sum(out["rho"][0] == out["max"][0]) >= 3


def test_single_lag_and_empty_bank():
    x = rng(13).standard_normal(M).astype(np.float32)
    p = small_bank()
    out = oracle.search(x, FS, p, M, want_rho=True)
    assert out["rho"].shape == (len(p["track"]), 1)
    empty = {k: v[:0] for k, v in p.items()}
    out = oracle.search(x, FS, empty, M)
    assert out["max"].shape == (0,)
    with pytest.raises(ValueError):
        oracle.search(x[:M - 1], FS, p, M)


# ----------------------------------------------------------------- templates

def test_template_unit_norm_support_and_reversal():
    for track in (oracle.LINEAR, oracle.POWERLAW):
        for D in (1.0, 0.45, 0.2):
            fs, Mt = 2048.0, 2048
            a = oracle.template(track, oracle.ASC, 55.0, 870.0, D, fs, Mt)
            d = oracle.template(track, oracle.DESC, 55.0, 870.0, D, fs, Mt)
            assert abs(np.sum(a * a) - 1.0) < 1e-13
            np.testing.assert_array_equal(d, a[::-1])
            MD = int(np.floor(D * fs + 0.5))
            ms = (Mt - MD) // 2
            assert oracle.support_len(D, fs) == MD
            nz = np.nonzero(a)[0]
            assert nz[0] >= ms and nz[-1] <= ms + MD - 1
            assert np.all(a[:ms] == 0) and np.all(a[ms + MD:] == 0)
            assert oracle.support_first(oracle.ASC, Mt, MD) == ms
            assert oracle.support_first(oracle.DESC, Mt, MD) == Mt - ms - MD


def test_butterfly_template_is_the_superposition_of_both_senses():
    """BOTH = (ascending + its time reverse), unit norm: it is symmetric in
    time and equals (h_asc + h_desc) / |h_asc + h_desc| because both have unit
    norm; its track paints both senses on the map."""
    for track in (oracle.LINEAR, oracle.POWERLAW):
        args = (track, 80.0, 700.0, 0.6, 2048.0, 2048)
        a = oracle.template(args[0], oracle.ASC, *args[1:])
        d = oracle.template(args[0], oracle.DESC, *args[1:])
        b = oracle.template(args[0], oracle.BOTH, *args[1:])
        ref = (a + d) / np.linalg.norm(a + d)
        np.testing.assert_allclose(b, ref, rtol=0, atol=1e-13)
        np.testing.assert_allclose(b, b[::-1], rtol=0, atol=1e-15)
        assert abs(np.sum(b * b) - 1.0) < 1e-13
    fs, Mt = 2048.0, 2048
    h = oracle.template(oracle.LINEAR, oracle.BOTH, 200.0, 600.0, 1.0, fs, Mt)
    x = np.zeros(3 * Mt, np.float32)
    x[500:500 + Mt] = h
    p = dict(track=np.array([0], np.int32), sense=np.array([oracle.BOTH], np.int32),
             f_lo=np.array([200.0]), f_hi=np.array([600.0]), D=np.array([1.0]))
    mp = oracle.search(x, fs, p, Mt, want_map=True)["map"]
    pa = dict(p, sense=np.array([oracle.ASC], np.int32))
    pd = dict(p, sense=np.array([oracle.DESC], np.int32))
    ha = oracle.template(oracle.LINEAR, oracle.ASC, 200.0, 600.0, 1.0, fs, Mt)
    # the map of the superposition holds an X: a rising and a falling track
    b = 500 + Mt // 4
    row = mp[int((b / fs) / 1e-3)]
    assert np.count_nonzero(row > 0.9) >= 2


def test_linear_template_phase_matches_scipy_chirp():
    fs, Mt, D, f0, f1 = 2048.0, 2048, 0.75, 120.0, 640.0
    h = oracle.template(oracle.LINEAR, oracle.ASC, f0, f1, D, fs, Mt)
    MD = int(np.floor(D * fs + 0.5))
    ms = (Mt - MD) // 2
    j = np.arange(MD)
    t = j / fs
    ref = np.sin(np.pi * (j + 0.5) / MD) ** 2 * scipy.signal.chirp(
        t, f0=f0, t1=D, f1=f1, method="linear", phi=0)
    ref /= np.linalg.norm(ref)
    np.testing.assert_allclose(h[ms:ms + MD], ref, rtol=0, atol=1e-12)


def test_powerlaw_instantaneous_frequency_follows_minus_three_eighths_law():
    fs, Mt, D, f0, f1 = 4096.0, 4096, 1.0, 40.0, 400.0
    h = oracle.template(oracle.POWERLAW, oracle.ASC, f0, f1, D, fs, Mt)
    MD = int(np.floor(D * fs + 0.5))
    ms = (Mt - MD) // 2
    seg = h[ms:ms + MD]
    ana = scipy.signal.hilbert(seg)
    ph = np.unwrap(np.angle(ana))
    finst = np.diff(ph) * fs / (2 * np.pi)
    t = (np.arange(MD - 1) + 0.5) / fs
    tc = D / (1 - (f0 / f1) ** (8.0 / 3.0))
    law = f0 * (1 - t / tc) ** (-3.0 / 8.0)
    mid = slice(int(0.15 * MD), int(0.85 * MD))
    rel = np.abs(finst[mid] - law[mid]) / law[mid]
    assert np.median(rel) < 2e-3 and np.max(rel) < 3e-2
    # end points of the track and t_c
    assert abs(oracle.freq(oracle.POWERLAW, f0, f1, D, 0.0) - f0) < 1e-12
    assert abs(oracle.freq(oracle.POWERLAW, f0, f1, D, D) - f1) < 1e-9
    # the end of the sweep is f_hi exactly, on both tracks (the map's cell edge
    # at f_hi / df must not depend on the last bit of a pow)
    for track in (oracle.LINEAR, oracle.POWERLAW):
        assert oracle.freq(track, 364.7022859372599, 900.0, 0.9033323293453285, 0.9033323293453285) == 900.0
        assert oracle.freq(track, f0, f1, D, D) == f1
    assert abs(oracle.powerlaw_tc(f0, f1, D) - tc) < 1e-12


def test_cycles_are_integral_of_frequency():
    for track in (oracle.LINEAR, oracle.POWERLAW):
        f0, f1, D = 33.0, 777.0, 0.6
        for t in np.linspace(0.01, D - 0.01, 7):
            e = 1e-6
            dc = (oracle.cycles(track, f0, f1, D, t + e) - oracle.cycles(track, f0, f1, D, t - e)) / (2 * e)
            assert abs(dc - oracle.freq(track, f0, f1, D, t)) < 1e-5 * f1
        assert oracle.cycles(track, f0, f1, D, 0.0) == 0.0


def test_zero_crossings_count_cycles():
    fs, Mt, D, f0, f1 = 2048.0, 2048, 1.0, 200.0, 600.0
    for track in (oracle.LINEAR, oracle.POWERLAW):
        h = oracle.template(track, oracle.ASC, f0, f1, D, fs, Mt)
        MD = int(np.floor(D * fs + 0.5))
        ms = (Mt - MD) // 2
        seg = h[ms:ms + MD]
        zc = np.sum(np.signbit(seg[1:]) != np.signbit(seg[:-1]))
        c = oracle.cycles(track, f0, f1, D, (MD - 1) / fs)
        assert abs(zc - 2 * c) <= 2


def test_invalid_chirps_rejected():
    ok = (oracle.LINEAR, oracle.ASC, 50.0, 900.0, 1.0, 2048.0, 2048)
    assert oracle.check_chirp(*ok)
    bad = [
        (oracle.LINEAR, oracle.ASC, 50.0, 1024.0, 1.0, 2048.0, 2048),   # Nyquist
        (oracle.LINEAR, oracle.ASC, 0.0, 900.0, 1.0, 2048.0, 2048),     # f_lo <= 0
        (oracle.LINEAR, oracle.ASC, 900.0, 50.0, 1.0, 2048.0, 2048),    # f_hi <= f_lo
        (oracle.LINEAR, oracle.ASC, 50.0, 900.0, 1.5, 2048.0, 2048),    # D*fs > M
        (oracle.LINEAR, oracle.ASC, 50.0, 900.0, 0.0, 2048.0, 2048),    # D <= 0
        (7, oracle.ASC, 50.0, 900.0, 1.0, 2048.0, 2048),
    ]
    for b in bad:
        assert not oracle.check_chirp(*b)
        with pytest.raises(ValueError):
            oracle.template(*b)


# ----------------------------------------------------------------- grid

def test_grid_counts_order_and_ranges():
    g = oracle.grid([oracle.LINEAR, oracle.POWERLAW], [oracle.ASC, oracle.DESC],
                    [0.2 + 0.1 * i for i in range(9)], 20.0, 1000.0, 6, 4)
    K = 2 * 2 * 9 * 6 * 4
    assert len(g["track"]) == K
    # bank index order: track, sense, duration, i, j (j fastest)
    k = ((((1 * 2 + 0) * 9 + 4) * 6 + 3) * 4 + 2)
    assert g["track"][k] == oracle.POWERLAW and g["sense"][k] == oracle.ASC
    assert abs(g["D"][k] - 0.6) < 1e-12
    assert abs(g["f_lo"][k] - (20.0 + 980.0 * 3 / 6)) < 1e-12
    lo = g["f_lo"][k]
    assert abs(g["f_hi"][k] - (lo + (1000.0 - lo) * 3 / 4)) < 1e-12
    assert np.all(g["f_hi"] > g["f_lo"]) and np.all(g["f_hi"] <= 1000.0 + 1e-9)
    # last j reaches f_max
    assert np.allclose(g["f_hi"][3::4], 1000.0)
    # the counts quoted for the paper-sized banks
    assert 2 * 2 * 9 * 600 * 400 == 8_640_000
    assert 2 * 512 * 1024 == 1 << 20


# ----------------------------------------------------------------- histogram

def test_histogram_matches_numpy():
    v = rng(14).uniform(0, 1, 5000)
    v[:3] = [0.0, 1.0, 0.5]
    c = oracle.histogram(v, 1024)
    ref, _ = np.histogram(v, bins=1024, range=(0.0, 1.0))
    np.testing.assert_array_equal(c, ref)
    assert c.sum() == len(v)


# ----------------------------------------------------------------- control

def test_splitmix64_published_values():
    with open(os.path.join(GOLDEN, "splitmix64.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        z = int(case["state"], 16)
        for out in case["outputs"]:
            # the published generator adds the golden gamma before mixing;
            # successive outputs come from successive states
            assert oracle.splitmix64(z) == int(out, 16)
            z = (z + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF


def test_permutation_keeps_histogram_and_is_bijective():
    x = rng(15).standard_normal(10007).astype(np.float32)
    y = oracle.permute(x, 4)
    np.testing.assert_array_equal(np.sort(y), np.sort(x))    # bitwise multiset
    pi = oracle.permutation(len(x), 4)
    assert np.array_equal(np.sort(pi), np.arange(len(x)))
    np.testing.assert_array_equal(y, x[pi])
    np.testing.assert_array_equal(oracle.permute(x, 4), y)   # deterministic
    assert not np.array_equal(oracle.permute(x, 5), y)
    # pi sorts the keys
    keys = np.array([oracle.splitmix64(4 ^ int(i)) for i in pi], dtype=np.uint64)
    assert np.all(keys[1:] >= keys[:-1])
    assert oracle.permute(x[:0], 4).shape == (0,)


def test_permutation_destroys_chirp_but_not_statistics():
    cfgx = np.zeros(4 * M, np.float32)
    h = oracle.template(oracle.LINEAR, oracle.ASC, 100.0, 400.0, 0.2, FS, M)
    cfgx[M:2 * M] = 50 * h
    cfgx += rng(16).standard_normal(4 * M).astype(np.float32)
    p = oracle.grid([oracle.LINEAR], [oracle.ASC], [0.2], 100.0, 400.0, 1, 1)
    p["f_hi"][:] = 400.0
    a = oracle.search(cfgx, FS, p, M)
    b = oracle.search(oracle.permute(cfgx, 9), FS, p, M)
    assert a["max"][0] > 0.8 and b["max"][0] < 0.4


# ----------------------------------------------------------------- TF map

def test_tf_map_paints_injected_track():
    fs, Mt, D, f0, f1 = 2048.0, 2048, 1.0, 200.0, 600.0
    dt, df = 1e-3, 4.0
    for sense in (oracle.ASC, oracle.DESC):
        h = oracle.template(oracle.LINEAR, sense, f0, f1, D, fs, Mt)
        n0 = 1000
        x = np.zeros(3 * Mt, np.float32)
        x[n0:n0 + Mt] = h
        p = dict(track=np.array([oracle.LINEAR], np.int32), sense=np.array([sense], np.int32),
                 f_lo=np.array([f0]), f_hi=np.array([f1]), D=np.array([D]))
        out = oracle.search(x, fs, p, Mt, kappa=5.0, dt=dt, df=df, want_map=True)
        mp = out["map"]
        assert out["argmax"][0] == n0 and abs(mp.max() - 1.0) < 1e-6
        t0 = n0 / fs
        hits = 0
        for b in range(mp.shape[0]):
            tb = (b + 0.5) * dt
            if not (t0 <= tb < t0 + D):
                continue
            t = tb - t0
            u = t if sense == oracle.ASC else D - t
            f = f0 + (f1 - f0) * u / D
            fb = int(np.floor(f / df))
            assert mp[b, fb] > 1.0 - 1e-6, (b, fb)
            hits += 1
        assert hits >= 995
        # nothing is painted outside the band swept by the track
        assert np.all(mp[:, : int(f0 // df) - 1] == 0)
        assert np.all(mp[:, int(f1 // df) + 2:] == 0)


# ----------------------------------------------------------------- Parseval predictor

def test_parseval_identity_for_circular_correlation():
    """For one segment of exactly F samples, sum_f |X|^2 |H|^2 / F equals the
    sum over all circular lags of the squared circular correlation."""
    r = rng(20)
    Mp = 64
    F = 2 * Mp
    x = r.standard_normal(F)
    h = r.standard_normal(Mp)
    P = oracle.welch_power(x, F)
    Hf = np.abs(np.fft.fft(h, F)) ** 2
    hpad = np.concatenate([h, np.zeros(F - Mp)])
    circ = [np.dot(np.roll(x, -t), hpad) for t in range(F)]
    assert abs(np.sum(P * Hf) / F - np.sum(np.square(circ))) < 1e-9 * np.sum(np.square(circ))


def test_parseval_sigma_white_noise_is_one_over_sqrt_m():
    Mw = 256
    h = oracle.template(oracle.LINEAR, oracle.ASC, 40.0, 400.0, 0.25, 1024.0, Mw)
    x = rng(21).standard_normal(Mw * 2000)
    s = oracle.parseval_sigma(x, h[None, :])[0]
    assert abs(s * np.sqrt(Mw) - 1.0) < 0.02
    # scale invariance and the all-zero series
    assert abs(oracle.parseval_sigma(3.0 * x, h[None, :])[0] - s) < 1e-12
    assert oracle.parseval_sigma(np.zeros(4 * Mw), h[None, :])[0] == 0.0


def test_parseval_sigma_is_exact_for_one_segment_of_circular_correlations():
    """For a series of exactly F = PARSEVAL_F samples (one Welch segment),
    sigma^2 F M sigma_x^2 equals the sum of the squared circular correlations
    of the series with the zero-padded template over all F lags (Parseval),
    computed here by plain loops over lags; templates longer than F/2 are
    refused."""
    F = oracle.PARSEVAL_F
    r = rng(24)
    x = r.standard_normal(F)
    Mp = 300
    h = r.standard_normal(Mp)
    h /= np.linalg.norm(h)
    s = oracle.parseval_sigma(x, h[None, :])[0]
    xx = np.concatenate([x, x[:Mp]])                # circular: the series wraps around
    circ = np.array([np.dot(xx[t:t + Mp], h) for t in range(F)])
    lhs = s * s * F * Mp * np.mean(x * x)
    assert abs(lhs - np.sum(circ ** 2)) < 1e-9 * np.sum(circ ** 2)
    with pytest.raises(ValueError):
        oracle.parseval_sigma(x, np.ones((1, F // 2 + 1)))


def test_parseval_sigma_predicts_measured_sigma_of_coloured_noise():
    """On stationary coloured noise the prediction agrees with the rms of rho
    measured by the search, template by template, to within the bias of a
    predictor: rho divides by the local window norm, whose fluctuations on red
    noise make E[C^2 / E_w] exceed E[C^2] / E[E_w] (here by ~5 %).  A
    low-frequency template sees several times the noise of a high-frequency
    one."""
    fs, Mw = 1024.0, 256
    p = oracle.grid([oracle.LINEAR], [oracle.ASC], [0.25], 10.0, 500.0, 2, 2)
    r = rng(22)
    w = r.standard_normal(Mw * 400)
    X = np.fft.rfft(w)
    f = np.fft.rfftfreq(len(w), 1 / fs)
    X *= 1.0 / np.maximum(f / 30.0, 0.2)            # red spectrum below 30 Hz
    x = np.fft.irfft(X, len(w)).astype(np.float32)
    H = oracle.bank(p, fs, Mw)
    pred = oracle.parseval_sigma(x, H)
    meas = oracle.search(x, fs, p, Mw)["sigma"]
    np.testing.assert_allclose(pred, meas, rtol=0.10)
    assert np.all(pred <= meas)                     # the bias has this sign
    assert pred.max() > 2 * pred.min()


def test_per_template_thresholds_paint_only_their_tails():
    fs, Mw = 1024.0, 256
    p = oracle.grid([oracle.LINEAR], [oracle.ASC, oracle.DESC], [0.25], 40.0, 400.0, 1, 2)
    x = rng(23).standard_normal(Mw * 8).astype(np.float32)
    out = oracle.search(x, fs, p, Mw, want_rho=True)
    K = len(p["track"])
    thr_k = np.array([0.15, 10.0, 0.15, 10.0])[:K]
    m1 = oracle.search(x, fs, p, Mw, thr_k=thr_k, want_map=True)["map"]
    only = {k: v[[0, 2]] for k, v in p.items()} if K == 4 else p
    m2 = oracle.search(x, fs, only, Mw, thr=0.15, want_map=True)["map"]
    np.testing.assert_array_equal(m1, m2)


# ----------------------------------------------------------------- skew-normal fit

def test_skewnorm_fit_recovers_known_parameters():
    """Samples of scipy's skew-normal with known (xi, omega, alpha) give back
    those parameters within their sampling error."""
    for alpha, xi, omega in ((4.0, 0.10, 0.02), (-3.0, 0.5, 0.1), (1.5, -1.0, 2.0)):
        v = scipy.stats.skewnorm.rvs(alpha, loc=xi, scale=omega, size=400_000,
                                     random_state=np.random.default_rng(int(abs(alpha) * 10)))
        f = oracle.skewnorm_fit(v)
        assert abs(f["xi"] - xi) < 0.02 * omega
        assert abs(f["omega"] / omega - 1.0) < 0.02
        assert abs(f["alpha"] / alpha - 1.0) < 0.1
        ref_skew = scipy.stats.skew(v)
        assert abs(f["skewness"] - ref_skew) < 1e-9


def test_skewnorm_fit_of_a_symmetric_sample_is_the_normal():
    """A sample symmetric about its mean has zero skewness, so the fit is the
    normal distribution: alpha = 0, xi = mean, omega = standard deviation."""
    u = np.random.default_rng(3).normal(0.0, 0.5, 100_000)
    v = np.concatenate([2.0 + u, 2.0 - u])
    f = oracle.skewnorm_fit(v)
    assert abs(f["skewness"]) < 1e-12 and abs(f["alpha"]) < 1e-3
    assert abs(f["xi"] - 2.0) < 1e-3 * 0.5 and abs(f["omega"] - np.std(v)) < 1e-9


def test_skewnorm_fit_clips_at_the_maximum_skewness():
    """An exponential sample (skewness 2) lies beyond the skew-normal's range;
    the fit saturates at |delta| -> 1 with a large positive alpha."""
    v = np.random.default_rng(4).exponential(1.0, 100_000)
    f = oracle.skewnorm_fit(v)
    assert f["skewness"] == pytest.approx(0.99527) and f["alpha"] > 20


# ----------------------------------------------------------------- coincidence pseudo-spectra

def _cells(nt, nf, cells):
    m = np.zeros((nt, nf), np.float32)
    for t, c in cells:
        m[t, c] = 0.5
    return m


def test_coincidence_hand_worked_example():
    """Counts worked out by hand: df = 4 Hz and delta_f = 8 Hz give a window
    of two cells; with dt = 0 only equal time cells pair, with dt = 1 the
    neighbouring rows too."""
    a = _cells(6, 10, [(1, 2), (3, 5), (5, 9)])
    b = _cells(6, 10, [(1, 4), (4, 7), (5, 6)])
    r = oracle.coincidence(a, b, 4.0, 8.0, 0)
    # a(1,2)-b(1,4): |2-4| = 2 <= 2 yes; a(3,5): row 3 of b empty; a(5,9)-b(5,6): 3 > 2 no
    assert r["indep_a"].tolist() == [0, 0, 1, 0, 0, 1, 0, 0, 0, 1]
    assert r["coinc_a"].tolist() == [0, 0, 1, 0, 0, 0, 0, 0, 0, 0]
    assert r["coinc_b"].tolist() == [0, 0, 0, 0, 1, 0, 0, 0, 0, 0]
    r = oracle.coincidence(a, b, 4.0, 8.0, 1)
    # now a(3,5)-b(4,7): |5-7| = 2 yes; a(5,9)-b(4,7): |9-7| = 2 yes; b(5,6) pairs
    # with neither a(5,9) (3 cells) nor a(3,5) (two rows away)
    assert r["coinc_a"].tolist() == [0, 0, 1, 0, 0, 1, 0, 0, 0, 1]
    assert r["coinc_b"].tolist() == [0, 0, 0, 0, 1, 0, 0, 1, 0, 0]
    r = oracle.coincidence(a, b, 4.0, 7.99, 1)          # one cell of window
    assert r["coinc_a"].sum() == 0 and r["coinc_b"].sum() == 0


def test_coincidence_special_cases():
    rng = np.random.default_rng(21)
    a = (rng.random((200, 64)) < 0.03) * rng.random((200, 64))
    b = (rng.random((200, 64)) < 0.03) * rng.random((200, 64))
    # a map against itself: every painted cell is simultaneous with itself
    r = oracle.coincidence(a, a, 4.0, 0.0, 0)
    np.testing.assert_array_equal(r["coinc_a"], r["indep_a"])
    np.testing.assert_array_equal(r["indep_a"], (a > 0).sum(axis=0))
    # exchanging the detectors exchanges the outputs
    r1, r2 = oracle.coincidence(a, b, 4.0, 50.0, 2), oracle.coincidence(b, a, 4.0, 50.0, 2)
    for x, y in (("indep_a", "indep_b"), ("coinc_a", "coinc_b")):
        np.testing.assert_array_equal(r1[x], r2[y])
    # disjoint in time: no coincidences
    a2, b2 = a.copy(), b.copy()
    a2[100:] = 0
    b2[:103] = 0
    r = oracle.coincidence(a2, b2, 4.0, 1000.0, 2)
    assert r["coinc_a"].sum() == 0 and r["coinc_b"].sum() == 0
    # counts grow with the windows and are bounded by the independent counts
    prev = None
    for w in (0.0, 8.0, 40.0, 400.0):
        r = oracle.coincidence(a, b, 4.0, w, 1)
        assert np.all(r["coinc_a"] <= r["indep_a"])
        if prev is not None:
            assert np.all(r["coinc_a"] >= prev)
        prev = r["coinc_a"]
    # an infinite window pairs every painted cell of a with any painted cell of b in reach in time
    r = oracle.coincidence(a, b, 4.0, 1e9, 0)
    rows_b = (b > 0).any(axis=1)
    np.testing.assert_array_equal(r["coinc_a"], ((a > 0) & rows_b[:, None]).sum(axis=0))


# ----------------------------------------------------------------- quadrature templates

def test_quadrature_partner_is_the_hilbert_transform():
    """The quadrature partner of a chirp well inside the band is the Hilbert
    transform of the template (the imaginary part of its analytic signal),
    up to the taper's edge effects, for either sense and for the
    superposition of both."""
    fs, M = 2048.0, 2048
    for track, sense, f0, f1, D in ((0, 0, 100.0, 600.0, 1.0), (1, 1, 80.0, 500.0, 0.8),
                                    (0, 2, 200.0, 300.0, 0.9)):
        hc = oracle.template(track, sense, f0, f1, D, fs, M, 0)
        hs = oracle.template(track, sense, f0, f1, D, fs, M, 1)
        hh = scipy.signal.hilbert(hc).imag
        c = np.dot(hh, hs) / np.linalg.norm(hh) / np.linalg.norm(hs)
        assert c > 0.999, (track, sense, c)
        assert abs(np.linalg.norm(hs) - 1.0) < 1e-12
        assert abs(np.dot(hc, hs)) < 0.02                       # nearly orthogonal
    # the superposition's pair is exactly orthogonal: symmetric against antisymmetric
    hc = oracle.template(0, 2, 200.0, 300.0, 0.9, fs, M, 0)
    hs = oracle.template(0, 2, 200.0, 300.0, 0.9, fs, M, 1)
    np.testing.assert_allclose(hs, -hs[::-1], atol=1e-15)
    assert abs(np.dot(hc, hs)) < 1e-12


def test_quadrature_output_is_phase_blind():
    """A noise-free signal cos(phi) h_c + sin(phi) h_s at a known offset gives
    a quadrature output of 1 there for every phase, up to the overlap
    eps = <h_c, h_s> of the pair; the cosine-only output follows cos(phi)."""
    fs, M = 1024.0, 1024
    p = dict(track=np.array([1], np.int32), sense=np.array([0], np.int32),
             f_lo=np.array([60.0]), f_hi=np.array([300.0]), D=np.array([0.9]))
    hc = oracle.template(1, 0, 60.0, 300.0, 0.9, fs, M, 0)
    hs = oracle.template(1, 0, 60.0, 300.0, 0.9, fs, M, 1)
    eps = abs(np.dot(hc, hs))
    for phi in (0.0, 0.4, np.pi / 2, 2.5):
        x = np.zeros(3000, np.float64)
        x[700:700 + M] = np.cos(phi) * hc + np.sin(phi) * hs
        x = x.astype(np.float32)
        q = oracle.search(x, fs, p, M, want_rho=True, quadrature=True)
        c = oracle.search(x, fs, p, M, want_rho=True)
        assert abs(q["rho"][0, 700] - 1.0) <= 2 * eps + 1e-6, (phi, q["rho"][0, 700])
        assert abs(c["rho"][0, 700] - np.cos(phi)) <= 2 * eps + 1e-6
        assert np.all(q["rho"][0] >= np.abs(c["rho"][0]) - 1e-12)
        assert q["argmax"][0] == 700


def test_quadrature_white_noise_second_moment():
    """For iid Gaussian windows E rho_cos^2 = E rho_sin^2 = 1/M exactly, so
    the mean of the quadrature output squared is 2/M."""
    rng = np.random.default_rng(17)
    fs, M = 512.0, 512
    spec = {"tracks": [0, 1], "senses": [0, 1], "durations": [0.9], "f_min": 20.0,
            "f_max": 250.0, "I": 3, "J": 3}
    p = oracle.grid(spec["tracks"], spec["senses"], spec["durations"], spec["f_min"],
                    spec["f_max"], spec["I"], spec["J"])
    x = rng.standard_normal(40000).astype(np.float32)
    q = oracle.search(x, fs, p, M, quadrature=True)
    m2 = np.mean(q["sigma"] ** 2)
    # 36 templates x 39489 correlated lags: a few % statistical spread
    assert abs(m2 * M / 2.0 - 1.0) < 0.05, m2 * M / 2
    assert q["thr"] == pytest.approx(5.0 * np.sqrt(2.0 / M))
