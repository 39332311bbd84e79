"""FP64 CPU oracle of the butterfly-filtering hot path (arXiv:1802.01685,
Sect. 2.1-2.2): chirp templates, bank grid, normalised sliding correlation,
per-template max/argmax/sigma, max-histogram, time-frequency map and the
time-randomised control.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and never imports it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over templates);
this module only compiles it with gcc and marshals numpy arrays through ctypes.
Every definition is a reading of the paper's prose; ``oracle.c`` states each
one next to the code.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LINEAR, POWERLAW = 0, 1
ASC, DESC, BOTH = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        d, l, i, p = C.c_double, C.c_long, C.c_int, C.c_void_p
        lib.oracle_powerlaw_tc.restype = d
        lib.oracle_powerlaw_tc.argtypes = [d, d, d]
        lib.oracle_cycles.restype = d
        lib.oracle_cycles.argtypes = [i, d, d, d, d]
        lib.oracle_freq.restype = d
        lib.oracle_freq.argtypes = [i, d, d, d, d]
        lib.oracle_support_len.restype = l
        lib.oracle_support_len.argtypes = [d, d]
        lib.oracle_support_first.restype = l
        lib.oracle_support_first.argtypes = [i, l, l]
        lib.oracle_check_chirp.restype = i
        lib.oracle_check_chirp.argtypes = [i, i, d, d, d, d, l]
        lib.oracle_template.restype = i
        lib.oracle_template.argtypes = [i, i, d, d, d, d, l, p]
        lib.oracle_template_phase.restype = i
        lib.oracle_template_phase.argtypes = [i, i, d, d, d, d, l, i, p]
        lib.oracle_grid.restype = l
        lib.oracle_grid.argtypes = [p, l, p, l, p, l, d, d, l, l, p, p, p, p, p]
        lib.oracle_correlate_raw.restype = None
        lib.oracle_correlate_raw.argtypes = [p, l, p, l, p, p]
        lib.oracle_search.restype = i
        lib.oracle_search.argtypes = [p, l, d, p, p, p, p, p, l, l, i, d, p, d, d, l, l,
                                      p, p, p, p, p]
        lib.oracle_histogram.restype = None
        lib.oracle_histogram.argtypes = [p, l, l, p]
        lib.oracle_splitmix64.restype = C.c_uint64
        lib.oracle_splitmix64.argtypes = [C.c_uint64]
        lib.oracle_permutation.restype = i
        lib.oracle_permutation.argtypes = [l, C.c_uint64, p]
        lib.oracle_permute.restype = i
        lib.oracle_permute.argtypes = [p, l, C.c_uint64, p]
        lib.oracle_num_threads.restype = i
        lib.oracle_num_threads.argtypes = []
        _lib = lib
        return lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


# ---------------------------------------------------------------- chirps

def powerlaw_tc(f_lo, f_hi, D):
    return _load().oracle_powerlaw_tc(f_lo, f_hi, D)


def cycles(track, f_lo, f_hi, D, t):
    return _load().oracle_cycles(track, f_lo, f_hi, D, t)


def freq(track, f_lo, f_hi, D, t):
    return _load().oracle_freq(track, f_lo, f_hi, D, t)


def support_len(D, fs):
    return _load().oracle_support_len(D, fs)


def support_first(sense, M, MD):
    return _load().oracle_support_first(sense, M, MD)


def check_chirp(track, sense, f_lo, f_hi, D, fs, M) -> bool:
    return _load().oracle_check_chirp(track, sense, f_lo, f_hi, D, fs, M) == 0


def template(track, sense, f_lo, f_hi, D, fs, M, phase: int = 0) -> np.ndarray:
    """Unit-norm template; phase 1 is the quadrature (sine-phase) partner."""
    h = np.zeros(M, np.float64)
    if _load().oracle_template_phase(track, sense, f_lo, f_hi, D, fs, M, int(phase), _ptr(h)):
        raise ValueError("invalid chirp parameters")
    return h


def grid(tracks, senses, durations, f_min, f_max, I, J) -> dict:
    tr = np.ascontiguousarray(tracks, np.int32)
    se = np.ascontiguousarray(senses, np.int32)
    du = np.ascontiguousarray(durations, np.float64)
    K = len(tr) * len(se) * len(du) * I * J
    out = dict(track=np.zeros(K, np.int32), sense=np.zeros(K, np.int32),
               f_lo=np.zeros(K), f_hi=np.zeros(K), D=np.zeros(K))
    n = _load().oracle_grid(_ptr(tr), len(tr), _ptr(se), len(se), _ptr(du), len(du),
                            f_min, f_max, I, J, _ptr(out["track"]), _ptr(out["sense"]),
                            _ptr(out["f_lo"]), _ptr(out["f_hi"]), _ptr(out["D"]))
    assert n == K
    return out


def bank(params: dict, fs: float, M: int, phase: int = 0) -> np.ndarray:
    """[K, M] FP64 templates in bank order (phase 1: their quadrature partners)."""
    K = len(params["track"])
    H = np.zeros((K, M), np.float64)
    for k in range(K):
        H[k] = template(int(params["track"][k]), int(params["sense"][k]),
                        float(params["f_lo"][k]), float(params["f_hi"][k]),
                        float(params["D"][k]), fs, M, phase)
    return H


# ---------------------------------------------------------------- correlation

def correlate_raw(x: np.ndarray, h: np.ndarray):
    x = np.ascontiguousarray(x, np.float32)
    h = np.ascontiguousarray(h, np.float64)
    L = len(x) - len(h) + 1
    num = np.zeros(L)
    en = np.zeros(L)
    _load().oracle_correlate_raw(_ptr(x), len(x), _ptr(h), len(h), _ptr(num), _ptr(en))
    return num, en


def map_shape(N: int, fs: float, dt: float, df: float):
    """Time bins cover the series, frequency bins cover [0, fs/2)."""
    nt = int(np.ceil(N / (fs * dt)))
    nf = int(np.ceil((fs / 2.0) / df))
    return nt, nf


def search(x: np.ndarray, fs: float, params: dict, M: int, *, kappa: float = 5.0,
           thr: float | None = None, thr_k: np.ndarray | None = None, dt: float = 1e-3,
           df: float = 4.0, want_rho: bool = False, want_map: bool = False,
           quadrature: bool = False) -> dict:
    """Full oracle search of one series against the bank given by ``params``.
    The map is painted by tails |rho| >= thr (default kappa / sqrt(M), or
    kappa sqrt(2 / M) for quadrature output), or >= thr_k[k] per template
    when thr_k is given.  With ``quadrature`` the output of template k is
    sqrt(rho_cos^2 + rho_sin^2), rho_sin from its sine-phase partner."""
    x = np.ascontiguousarray(x, np.float32)
    N = len(x)
    K = len(params["track"])
    L = N - M + 1
    if thr is None:
        thr = kappa * np.sqrt((2.0 if quadrature else 1.0) / M)
    tr = np.ascontiguousarray(params["track"], np.int32)
    se = np.ascontiguousarray(params["sense"], np.int32)
    fl = np.ascontiguousarray(params["f_lo"], np.float64)
    fh = np.ascontiguousarray(params["f_hi"], np.float64)
    Dd = np.ascontiguousarray(params["D"], np.float64)
    nt, nf = map_shape(N, fs, dt, df)
    rho = np.zeros((K, L)) if want_rho else None
    vmax = np.zeros(K)
    arg = np.zeros(K, np.int64)
    sig = np.zeros(K)
    mp = np.zeros((nt, nf)) if want_map else None
    tk = np.ascontiguousarray(thr_k, np.float64) if thr_k is not None else None
    rc = _load().oracle_search(_ptr(x), N, fs, _ptr(tr), _ptr(se), _ptr(fl), _ptr(fh),
                               _ptr(Dd), K, M, int(bool(quadrature)), float(thr), _ptr(tk), dt, df,
                               nt, nf, _ptr(rho),
                               _ptr(vmax), _ptr(arg), _ptr(sig), _ptr(mp))
    if rc:
        raise ValueError("oracle_search: invalid input")
    return dict(rho=rho, max=vmax, argmax=arg, sigma=sig, map=mp, thr=float(thr),
                nt=nt, nf=nf)


def welch_power(x: np.ndarray, F: int) -> np.ndarray:
    """Averaged periodogram of x over rectangular segments of F samples at hop
    F/2, all F DFT bins: P(f) = mean_s |DFT_F(x_s)(f)|^2.  A series shorter than
    F is one zero-padded segment scaled by F/N.  (Predictor step of Sect. 2.2
    and Fig. 5: sigma of the filter output from Parseval's theorem.)"""
    x = np.asarray(x, np.float64)
    N = len(x)
    if N >= F:
        hop = F // 2
        S = (N - F) // hop + 1
        P = np.zeros(F)
        for s in range(S):
            P += np.abs(np.fft.fft(x[s * hop:s * hop + F])) ** 2
        return P / S
    return np.abs(np.fft.fft(x, F)) ** 2 * (F / N)


# DFT length and Welch segment length of the Parseval predictor: 16384
# samples, the real segment of the FFT route (the paper's predictor works on
# the segment transforms of its FFT route; it gives no length)
PARSEVAL_F = 16384


def parseval_sigma(x: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Predicted standard deviation of rho for each template row of H ([K, M]),
    before the search, from Parseval's theorem (Sect. 2.2, Fig. 5 caption):
      E[C_k(tau)^2] = sum_f S_x(f) |H_k(f)|^2 / F   (S_x = P / F, F = PARSEVAL_F),
      rho = C / |window|,  |window|^2 ~ M sigma_x^2,
    so sigma_k^2 = sum_f P(f) |H_k(f)|^2 / (F^2 M sigma_x^2), the sum over all
    F bins, sigma_x^2 the mean of x^2; 0 for an all-zero series.  F >= 2M
    keeps the template's circular autocorrelation free of wrap-around, so
    templates of at most F/2 samples."""
    H = np.atleast_2d(np.asarray(H, np.float64))
    K, M = H.shape
    F = PARSEVAL_F
    if 2 * M > F:
        raise ValueError("parseval_sigma: templates longer than F/2")
    x = np.asarray(x, np.float64)
    sx2 = np.mean(x * x)
    if sx2 == 0.0:
        return np.zeros(K)
    P = welch_power(x, F)
    out = np.zeros(K)
    for k in range(K):
        Hf = np.abs(np.fft.fft(H[k], F)) ** 2
        out[k] = np.sqrt(np.sum(P * Hf) / (F * F * M * sx2))
    return out


def skewnorm_fit(v: np.ndarray) -> dict:
    """Skew-normal fit of the per-template maxima (Fig. 2: the distributions of
    maxima are left-truncated skewed Gaussians) by the method of moments of
    Azzalini (1985): from the sample mean m, standard deviation s and skewness
    g (clipped to the skew-normal's range |g| < 0.99527),
      |delta| = sqrt(pi/2 * |g|^(2/3) / (|g|^(2/3) + ((4 - pi)/2)^(2/3))),
      alpha = delta / sqrt(1 - delta^2),
      omega = s / sqrt(1 - 2 delta^2 / pi),  xi = m - omega delta sqrt(2/pi).
    Moments use the population (1/n) normalisation; the truncation is not
    modelled."""
    v = np.asarray(v, np.float64)
    n = len(v)
    m = v.mean()
    d = v - m
    var = np.mean(d * d)
    sd = np.sqrt(var)
    g = np.mean(d ** 3) / var ** 1.5 if var > 0 else 0.0
    gmax = 0.99527
    g = float(np.clip(g, -gmax, gmax))
    a = abs(g) ** (2.0 / 3.0)
    delta = np.sign(g) * np.sqrt(np.pi / 2.0 * a / (a + ((4.0 - np.pi) / 2.0) ** (2.0 / 3.0)))
    alpha = delta / np.sqrt(1.0 - delta * delta)
    omega = sd / np.sqrt(1.0 - 2.0 * delta * delta / np.pi)
    xi = m - omega * delta * np.sqrt(2.0 / np.pi)
    return dict(n=n, mean=m, sd=sd, skewness=g, xi=xi, omega=omega, alpha=alpha)


def coincidence(map_a: np.ndarray, map_b: np.ndarray, df: float, delta_f_hz: float,
                dt_cells: int = 0) -> dict:
    """Pseudo-spectra of tails of two detectors (Fig. 6): per frequency cell
    c of two time-frequency maps, the independent counts of time cells that
    a tail painted, and the simultaneous counts of those that have a painted
    cell of the other detector within dt_cells time cells and within
    delta_f_hz (|c - c'| df <= delta_f_hz, i.e. floor(delta_f_hz / df)
    cells).  The maps are cut to their common number of time cells.  Plain
    loops over the painted cells."""
    nt = min(map_a.shape[0], map_b.shape[0])
    nf = map_a.shape[1]
    oa = np.asarray(map_a[:nt]) > 0
    ob = np.asarray(map_b[:nt]) > 0
    w = int(np.floor(delta_f_hz / df + 1e-9))
    out = {k: np.zeros(nf, np.int64) for k in ("indep_a", "indep_b", "coinc_a", "coinc_b")}

    def any_in_window(o, t, c):
        t0, t1 = max(t - dt_cells, 0), min(t + dt_cells, nt - 1)
        c0, c1 = max(c - w, 0), min(c + w, nf - 1)
        return bool(o[t0:t1 + 1, c0:c1 + 1].any())

    for t, c in zip(*np.nonzero(oa)):
        out["indep_a"][c] += 1
        out["coinc_a"][c] += any_in_window(ob, t, c)
    for t, c in zip(*np.nonzero(ob)):
        out["indep_b"][c] += 1
        out["coinc_b"][c] += any_in_window(oa, t, c)
    return out


def histogram(v: np.ndarray, nbins: int = 1024) -> np.ndarray:
    v = np.ascontiguousarray(v, np.float64)
    c = np.zeros(nbins, np.uint32)
    _load().oracle_histogram(_ptr(v), len(v), nbins, _ptr(c))
    return c


# ---------------------------------------------------------------- control

def splitmix64(z: int) -> int:
    return int(_load().oracle_splitmix64(z & 0xFFFFFFFFFFFFFFFF))


def permutation(n: int, seed: int) -> np.ndarray:
    pi = np.zeros(max(n, 1), np.int64)
    if _load().oracle_permutation(n, seed & 0xFFFFFFFFFFFFFFFF, _ptr(pi)):
        raise MemoryError
    return pi[:n]


def permute(x: np.ndarray, seed: int) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    y = np.zeros(max(len(x), 1), np.float32)
    if _load().oracle_permute(_ptr(x), len(x), seed & 0xFFFFFFFFFFFFFFFF, _ptr(y)):
        raise MemoryError
    return y[:len(x)]


def num_threads() -> int:
    return int(_load().oracle_num_threads())
