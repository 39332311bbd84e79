"""Seeded synthetic inputs shaped like the paper's workloads.

The paper analyses LIGO strain at 4096 samples/s in 16 s segments (Fig. 5
caption), BeppoSAX light curves binned at 0.5 ms (Sect. 2.1) and banks of
0.5 M to 8.64 M one-second chirp templates (Sect. 2.1-2.2, Fig. 6).  None of
those data sets is available here, so every input is synthetic: numpy PCG64
streams with fixed seeds, generated once and fed unchanged to both the CUDA
library and the CPU oracle.

This module is shared by the tests, the benchmark and the smoke check.  It
holds no arithmetic of the method (no template bank, no correlation, no
normalisation, no permutation): the injected test signals are built here with
their own construction (frequency integrated numerically, Tukey taper, sine
phase), so they are data, not bank templates.  Bank grids are returned as plain
parameter lists; each side expands them with its own code.
"""
from __future__ import annotations

import numpy as np

# chirp-parameter codes shared with the C-ABI (plain enumerations; BOTH is
# the superposition of an ascending chirp and its time reverse)
LINEAR, POWERLAW = 0, 1
ASC, DESC, BOTH = 0, 1, 2


# ------------------------------------------------------------- test signals

def chirp_signal(f_start: float, f_end: float, D: float, fs: float,
                 law: str = "linear") -> np.ndarray:
    """Unit-norm injected chirp of duration D sweeping f_start -> f_end.

    ``law='linear'`` sweeps linearly; ``law='powerlaw'`` follows an
    inspiral-like f ~ (t_c - t)^(-3/8) rising from f_start to f_end.  The
    phase is the running sum of the sampled frequency; the envelope is a Tukey
    window with 10 % cosine tapers.
    """
    n = int(round(D * fs))
    t = np.arange(n, dtype=np.float64) / fs
    if law == "linear":
        f = f_start + (f_end - f_start) * t / D
    elif law == "powerlaw":
        if not f_end > f_start:
            raise ValueError("power-law test signal must ascend")
        tc = D / (1.0 - (f_start / f_end) ** (8.0 / 3.0))
        f = f_start * (1.0 - t / tc) ** (-3.0 / 8.0)
    else:
        raise ValueError(law)
    phase = np.cumsum(f) / fs
    alpha = 0.1
    w = np.ones(n)
    edge = int(alpha * n / 2)
    if edge > 0:
        ramp = 0.5 * (1.0 - np.cos(np.pi * np.arange(edge) / edge))
        w[:edge] = ramp
        w[n - edge:] = ramp[::-1]
    s = w * np.sin(2.0 * np.pi * phase)
    return s / np.sqrt(np.sum(s * s))


def inject(x: np.ndarray, s: np.ndarray, n0: int, amplitude: float) -> np.ndarray:
    y = x.astype(np.float64).copy()
    y[n0:n0 + len(s)] += amplitude * s
    return y


# ------------------------------------------------------------- noise models

def white(n: int, rng: np.random.Generator, sigma: float = 1.0) -> np.ndarray:
    return sigma * rng.standard_normal(n)


def gw_coloured(n: int, fs: float, rng: np.random.Generator,
                f_wall: float = 30.0) -> np.ndarray:
    """Gaussian noise with an f^-2 power wall below f_wall (amplitude ~ 1/f
    between 1 Hz and f_wall, flat above, no DC), rescaled to unit variance."""
    w = rng.standard_normal(n)
    W = np.fft.rfft(w)
    f = np.fft.rfftfreq(n, 1.0 / fs)
    amp = np.ones_like(f)
    low = f < f_wall
    amp[low] = f_wall / np.maximum(f[low], 1.0)
    amp[0] = 0.0
    y = np.fft.irfft(W * amp, n)
    return y / np.std(y)


def kolmogorov_field(n: int, fs: float, rng: np.random.Generator) -> np.ndarray:
    """Unit-variance Gaussian field with power spectrum ~ f^(-5/3) above 1/T."""
    w = rng.standard_normal(n)
    W = np.fft.rfft(w)
    f = np.fft.rfftfreq(n, 1.0 / fs)
    fmin = fs / n
    amp = np.where(f >= fmin, np.maximum(f, fmin) ** (-5.0 / 6.0), 0.0)
    y = np.fft.irfft(W * amp, n)
    return y / np.std(y)


def grb_lightcurve(n: int, fs: float, rng: np.random.Generator,
                   rate: float = 500.0, mod: float = 0.3) -> np.ndarray:
    """Mean-subtracted Poisson photon counts in bins of 1/fs seconds with rate
    rate * (1 + mod * g), g a Kolmogorov field."""
    g = kolmogorov_field(n, fs, rng)
    lam = np.clip(rate * (1.0 + mod * g) / fs, 0.0, None)
    c = rng.poisson(lam).astype(np.float64)
    return c - c.mean()


# ------------------------------------------------------------- bank grids

def grid_spec(tracks, senses, durations, f_min, f_max, I, J) -> dict:
    return dict(tracks=list(tracks), senses=list(senses),
                durations=[float(d) for d in durations], f_min=float(f_min),
                f_max=float(f_max), I=int(I), J=int(J))


def grid_size(spec: dict) -> int:
    return (len(spec["tracks"]) * len(spec["senses"]) * len(spec["durations"])
            * spec["I"] * spec["J"])


# ------------------------------------------------------------- workloads

def tiny(seed: int = 1, n: int = 8192, fs: float = 2048.0, I: int = 8, J: int = 16):
    """4 s of unit white noise at 2048 Hz with one descending linear chirp
    600 -> 200 Hz (1 s, SNR 8) at a seeded offset; bank of 2 x I x J linear
    1 s templates over [50, 1000] Hz, both senses (256 for I=8, J=16)."""
    rng = np.random.default_rng(seed)
    M = int(fs)
    x = white(n, rng)
    n0 = int(rng.integers(0, n - M + 1))
    s = chirp_signal(600.0, 200.0, 1.0, fs, "linear")
    x = inject(x, s, n0, 8.0).astype(np.float32)
    spec = grid_spec([LINEAR], [ASC, DESC], [1.0], 50.0, 1000.0, I, J)
    return dict(name="tiny", series=[x], fs=fs, M=M, grid=spec, n0=[n0])


def gw_pair(seeds=(2, 3), n: int = 262144, fs: float = 4096.0, I: int = 256,
            J: int = 256, amplitude: float = 8.0, inj_seed: int = 2):
    """Two 64 s coloured-noise series at 4096 Hz with a common power-law chirp
    40 -> 400 Hz (1 s) at the same seeded offset; bank of I x J ascending
    power-law 1 s templates over [40, 400] Hz (65,536 for I=J=256).  The
    time-randomised controls use permutation seeds 4 and 5."""
    M = int(fs)
    r0 = np.random.default_rng(inj_seed + 1000)
    n0 = int(r0.integers(0, n - M + 1))
    s = chirp_signal(40.0, 400.0, 1.0, fs, "powerlaw")
    xs = []
    for sd in seeds:
        rng = np.random.default_rng(sd)
        xs.append(inject(gw_coloured(n, fs, rng), s, n0, amplitude).astype(np.float32))
    spec = grid_spec([POWERLAW], [ASC], [1.0], 40.0, 400.0, I, J)
    return dict(name="gw_pair", series=xs, fs=fs, M=M, grid=spec, n0=[n0, n0],
                control_seeds=[4, 5])


def grb_batch(seed: int = 6, n_series: int = 42, fs: float = 2000.0,
              t_min: float = 20.0, t_max: float = 200.0, I: int = 512,
              J: int = 1024):
    """n_series mean-subtracted Poisson light curves at 0.5 ms bins, lengths
    uniform in [t_min, t_max] s; bank of 2 x I x J linear 1 s templates over
    [20, 999] Hz, both senses (1,048,576 for I=512, J=1024).  The band stops
    1 Hz short of 1000 Hz, the Nyquist frequency of 0.5 ms bins, which no
    template may reach."""
    rng = np.random.default_rng(seed)
    M = int(fs)
    lens = rng.uniform(t_min, t_max, n_series)
    xs = [grb_lightcurve(int(round(T * fs)), fs, rng).astype(np.float32) for T in lens]
    spec = grid_spec([LINEAR], [ASC, DESC], [1.0], 20.0, 999.0, I, J)
    return dict(name="grb_batch", series=xs, fs=fs, M=M, grid=spec)


def full_bank(seed: int = 7, n: int = 65536, fs: float = 2048.0, I: int = 600,
              J: int = 400, amplitude: float = 8.0):
    """32 s of unit white noise at 2048 Hz with three injected chirps (linear
    ascending, linear descending, power-law ascending); bank over both tracks,
    both senses and nine sweep times 0.2..1.0 s in [20, 1000] Hz
    (8,640,000 templates for I=600, J=400)."""
    rng = np.random.default_rng(seed)
    M = int(fs)
    x = white(n, rng)
    sigs = [chirp_signal(150.0, 450.0, 1.0, fs, "linear"),
            chirp_signal(700.0, 300.0, 0.6, fs, "linear"),
            chirp_signal(60.0, 250.0, 0.8, fs, "powerlaw")]
    n0 = []
    span = (n - M) // 3
    for i, s in enumerate(sigs):
        o = int(rng.integers(i * span, (i + 1) * span - len(s)))
        n0.append(o)
        x = inject(x, s, o, amplitude)
    durs = [0.2 + 0.1 * i for i in range(9)]
    spec = grid_spec([LINEAR, POWERLAW], [ASC, DESC], durs, 20.0, 1000.0, I, J)
    return dict(name="full_bank", series=[x.astype(np.float32)], fs=fs, M=M,
                grid=spec, n0=n0)


def serving_stream(seed: int = 8, n_requests: int = 200, rate_hz: float = 50.0,
                   t_min: float = 4.0, t_max: float = 256.0, k_min_log2: int = 12,
                   k_max_log2: int = 20):
    """Seeded Poisson arrival stream of search requests: series length uniform
    in [t_min, t_max] s, fs in {2048, 4096}, Gaussian or Poisson-count kind,
    bank slice of 2^u templates with u uniform in [k_min_log2, k_max_log2].
    Returns request descriptors; ``request_series`` materialises a series."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    t_arr = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(n_requests):
        reqs.append(dict(
            arrival_s=float(t_arr[i]),
            T_s=float(rng.uniform(t_min, t_max)),
            fs=float(rng.choice([2048.0, 4096.0])),
            kind=str(rng.choice(["gauss", "poisson"])),
            n_templates=int(2 ** int(rng.integers(k_min_log2, k_max_log2 + 1))),
            seed=int(rng.integers(0, 2 ** 31)),
        ))
    return reqs


def request_series(req: dict) -> np.ndarray:
    rng = np.random.default_rng(req["seed"])
    n = int(round(req["T_s"] * req["fs"]))
    if req["kind"] == "gauss":
        return white(n, rng).astype(np.float32)
    return grb_lightcurve(n, req["fs"], rng).astype(np.float32)
