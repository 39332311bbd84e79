"""The seeded synthetic inputs follow their stated recipes (CPU).

The workloads stand in for the paper's data (LIGO strain at 4096 Hz, BeppoSAX
light curves at 0.5 ms bins, banks of up to 8.64 M one-second chirps), so their
shapes, rates, spectra and bank sizes are checked here against the recipe each
generator states, by properties computed independently of the generator."""
import numpy as np

from paper_1802_01685_gb300 import synth


def zero_crossings(s):
    nz = s[s != 0]
    return int(np.count_nonzero(np.signbit(nz[1:]) != np.signbit(nz[:-1])))


def test_injected_chirps_sweep_their_band():
    """Unit norm, and a sine of phase 2 pi int f crosses zero twice per cycle:
    the linear sweep 600 -> 200 Hz over 1 s holds (600 + 200) / 2 = 400
    cycles; the power law f_lo (1 - t/t_c)^(-3/8) holds
    (8/5) f_lo t_c (1 - (1 - D/t_c)^(5/8)) cycles, its closed-form integral."""
    fs = 8192.0
    s = synth.chirp_signal(600.0, 200.0, 1.0, fs, "linear")
    assert abs(np.sum(s * s) - 1.0) < 1e-12
    assert abs(zero_crossings(s) - 2 * 400) <= 3
    f0, f1, D = 40.0, 400.0, 1.0
    s = synth.chirp_signal(f0, f1, D, fs, "powerlaw")
    tc = D / (1.0 - (f0 / f1) ** (8.0 / 3.0))
    cycles = 1.6 * f0 * tc * (1.0 - (1.0 - D / tc) ** 0.625)
    assert abs(zero_crossings(s) - 2 * cycles) <= 3
    # the frequency rises: more crossings in the last tenth than in the first
    n = len(s)
    assert zero_crossings(s[-n // 10:]) > 3 * zero_crossings(s[:n // 10])


def test_tiny_workload():
    w = synth.tiny()
    x, fs, M, n0 = w["series"][0], w["fs"], w["M"], w["n0"][0]
    assert x.dtype == np.float32 and len(x) == 8192 and fs == 2048.0 and M == 2048
    assert 0 <= n0 <= len(x) - M
    assert synth.grid_size(w["grid"]) == 256
    # the injected chirp projects with amplitude 8 on top of unit white noise
    s = synth.chirp_signal(600.0, 200.0, 1.0, fs, "linear")
    assert abs(float(np.dot(x[n0:n0 + len(s)].astype(np.float64), s)) - 8.0) < 5.0


def test_gw_pair_workload():
    """Two 64 s series at 4096 Hz, unit variance, no DC, a power wall with
    amplitude 30/f below 30 Hz: the mean power over 5-10 Hz is
    (1/5 Hz) int_5^10 (30/f)^2 df = 18 times the flat level above 30 Hz."""
    w = synth.gw_pair()
    fs = w["fs"]
    assert fs == 4096.0 and w["M"] == 4096 and w["control_seeds"] == [4, 5]
    assert synth.grid_size(w["grid"]) == 65536
    assert w["grid"]["tracks"] == [synth.POWERLAW] and w["grid"]["senses"] == [synth.ASC]
    assert w["n0"][0] == w["n0"][1]
    for x in w["series"]:
        assert x.dtype == np.float32 and len(x) == 262144
        x = x.astype(np.float64)
        assert abs(x.var() - 1.0) < 0.01
        assert abs(x.mean()) < 1e-3
        p = np.abs(np.fft.rfft(x)) ** 2
        f = np.fft.rfftfreq(len(x), 1.0 / fs)
        ratio = p[(f >= 5) & (f < 10)].mean() / p[(f >= 100) & (f < 1000)].mean()
        assert 14.0 < ratio < 22.0, ratio
    assert not np.array_equal(w["series"][0], w["series"][1])


def test_grb_batch_workload():
    """42 light curves of 20-200 s at 0.5 ms bins: mean-subtracted Poisson
    counts of about 500 photons/s, i.e. 0.25 per bin (a count of 0 sits at
    minus the mean), on the 2^20-template linear bank below Nyquist."""
    w = synth.grb_batch()
    fs = w["fs"]
    assert fs == 2000.0 and w["M"] == 2000 and len(w["series"]) == 42
    assert synth.grid_size(w["grid"]) == 2 ** 20 and w["grid"]["f_max"] < fs / 2
    lens = np.array([len(x) for x in w["series"]])
    assert lens.min() >= 20 * fs and lens.max() <= 200 * fs
    assert lens.max() - lens.min() > 100 * fs                   # the lengths really vary
    for x in w["series"][:6]:
        x = x.astype(np.float64)
        assert abs(x.mean()) < 1e-6
        mean_count = -x.min()
        assert 0.24 < mean_count < 0.26, mean_count
        counts = x + mean_count
        assert np.abs(counts - np.rint(counts)).max() < 1e-5   # whole photon counts


def test_full_bank_workload():
    w = synth.full_bank()
    x, fs, M = w["series"][0], w["fs"], w["M"]
    assert len(x) == 65536 and fs == 2048.0 and M == 2048
    g = w["grid"]
    assert synth.grid_size(g) == 8_640_000
    np.testing.assert_allclose(g["durations"], np.arange(2, 11) / 10.0, atol=1e-12)
    assert g["tracks"] == [synth.LINEAR, synth.POWERLAW] and g["senses"] == [synth.ASC, synth.DESC]
    span = (len(x) - M) // 3
    for i, o in enumerate(w["n0"]):
        assert i * span <= o < (i + 1) * span
    assert abs(x.astype(np.float64).var() - 1.0) < 0.05


def test_serving_stream():
    reqs = synth.serving_stream()
    assert len(reqs) == 200
    t = np.array([r["arrival_s"] for r in reqs])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert 0.8 / 50 < np.diff(t).mean() < 1.2 / 50               # Poisson arrivals at 50/s
    assert all(4.0 <= r["T_s"] <= 256.0 for r in reqs)
    assert {r["fs"] for r in reqs} == {2048.0, 4096.0}
    assert {r["kind"] for r in reqs} == {"gauss", "poisson"}
    ks = {r["n_templates"] for r in reqs}
    assert ks <= {2 ** u for u in range(12, 21)} and len(ks) >= 6
    x = synth.request_series(reqs[0])
    assert len(x) == int(round(reqs[0]["T_s"] * reqs[0]["fs"])) and x.dtype == np.float32


def test_inputs_are_deterministic():
    a, b = synth.tiny(), synth.tiny()
    np.testing.assert_array_equal(a["series"][0], b["series"][0])
    assert synth.serving_stream() == synth.serving_stream()
    assert not np.array_equal(synth.tiny(seed=2)["series"][0], a["series"][0])
