"""ctypes binding of the C ABI in include/bf.h (argument marshalling only).

Every function of the header is exposed under the same name and raises
``BFError`` when the call returns a status other than BF_OK (or one of the
statuses the caller asked to receive).  Arrays may be numpy arrays (host
memory) or torch tensors (their ``data_ptr()``; host or CUDA).  All arithmetic
runs in the CUDA library: if ``libbf.so`` is missing this module raises on
load -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# the library; BF_LIBRARY selects another build of it (libbf_debug.so)
LIB_PATH = os.environ.get("BF_LIBRARY") or os.path.join(_PKG, "libbf.so")

# ---------------------------------------------------------------- constants
BF_OK, BF_EINVAL, BF_ENOMEM, BF_ECUDA, BF_ETIMEDOUT, BF_EPENDING, BF_EAGAIN, \
    BF_ECANCELED, BF_EDEVICE, BF_ENOTSUP = range(10)
BF_LINEAR, BF_POWERLAW = 0, 1
BF_ASC, BF_DESC, BF_BOTH = 0, 1, 2
BF_FP32, BF_BF16, BF_SPLIT_BF16, BF_FFT_FP32, BF_SPLIT_FP16 = 0, 1, 2, 3, 4
BF_BANK_FP32, BF_BANK_SPLIT_BF16, BF_BANK_GENERATED, BF_BANK_QUADRATURE, BF_BANK_SPLIT_FP16 = 1, 2, 4, 8, 16
BF_SERVE_FAIR, BF_SERVE_SHORTEST = 0, 1
BF_SIGMA_WHITE, BF_SIGMA_PARSEVAL = 0, 1

PRECISIONS = {"fp32": BF_FP32, "bf16": BF_BF16, "split_bf16": BF_SPLIT_BF16, "fft_fp32": BF_FFT_FP32,
              "split_fp16": BF_SPLIT_FP16}


class BFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"bf status {status}: {msg}")
        self.status = status


# ---------------------------------------------------------------- structs
class bf_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("hbm_budget", C.c_size_t),
                ("max_candidates", C.c_size_t), ("serve_slots", C.c_int32),
                ("serve_queue", C.c_int32), ("log_level", C.c_int32), ("serve_policy", C.c_int32)]


class bf_chirp(C.Structure):
    _fields_ = [("track", C.c_int32), ("sense", C.c_int32), ("f_lo", C.c_double),
                ("f_hi", C.c_double), ("sweep_s", C.c_double)]


class bf_chirp_grid(C.Structure):
    _fields_ = [("tracks", C.POINTER(C.c_int32)), ("n_tracks", C.c_size_t),
                ("senses", C.POINTER(C.c_int32)), ("n_senses", C.c_size_t),
                ("durations", C.POINTER(C.c_double)), ("n_durations", C.c_size_t),
                ("f_min", C.c_double), ("f_max", C.c_double), ("I", C.c_size_t),
                ("J", C.c_size_t)]


class bf_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("bank_begin", C.c_size_t),
                ("bank_end", C.c_size_t), ("kappa", C.c_double), ("map_dt_s", C.c_double),
                ("map_df_hz", C.c_double), ("want_map", C.c_int32), ("want_hist", C.c_int32),
                ("hist_bins", C.c_uint32), ("stream", C.c_void_p), ("rho_out", C.c_void_p),
                ("want_tails", C.c_int32), ("tail_sigma", C.c_int32), ("tile_lags", C.c_int32)]


class bf_tail(C.Structure):
    _fields_ = [("series", C.c_uint32), ("k", C.c_uint32), ("tau", C.c_uint32), ("rho", C.c_float)]


class bf_result_info(C.Structure):
    _fields_ = [("n_series", C.c_size_t), ("n_templates", C.c_size_t),
                ("template_len", C.c_size_t), ("correlations", C.c_double),
                ("useful_flops", C.c_double), ("n_candidates", C.c_uint64),
                ("candidates_overflow", C.c_int32), ("threshold", C.c_float),
                ("hist_bins", C.c_uint32), ("kernel_ms", C.c_double), ("tile_lags", C.c_int32)]


class bf_skewnorm(C.Structure):
    _fields_ = [("n", C.c_double), ("mean", C.c_double), ("sd", C.c_double),
                ("skewness", C.c_double), ("xi", C.c_double), ("omega", C.c_double),
                ("alpha", C.c_double)]


BF_FIT_MEAN = (1 << 64) - 1


class bf_request(C.Structure):
    _fields_ = [("series", C.c_void_p), ("n", C.c_size_t), ("fs", C.c_double),
                ("bank", C.c_void_p), ("opts", bf_opts)]


class bf_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64),
                ("cancelled", C.c_uint64), ("rejected", C.c_uint64), ("queued", C.c_uint64),
                ("active", C.c_uint64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("correlations_per_s", C.c_double), ("launches", C.c_uint64),
                ("hbm_in_use", C.c_size_t)]


# ---------------------------------------------------------------- loading
_lock = threading.Lock()
_lib = None


def load() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run "
                               "__graft_entry__.build() (no CPU fallback exists)")
        lib = C.CDLL(LIB_PATH)
        p, s, i, d, u64 = C.c_void_p, C.c_size_t, C.c_int, C.c_double, C.c_uint64
        P = C.POINTER
        sig = {
            "bf_config_default": (None, [P(bf_config)]),
            "bf_init": (i, [P(bf_config), P(p)]),
            "bf_destroy": (None, [p]),
            "bf_bank_create": (i, [p, P(bf_chirp), s, d, d, C.c_uint, P(p)]),
            "bf_bank_create_grid": (i, [p, P(bf_chirp_grid), d, d, C.c_uint, P(p)]),
            "bf_bank_destroy": (None, [p]),
            "bf_bank_size": (s, [p]),
            "bf_bank_template_len": (s, [p]),
            "bf_bank_rows": (s, [p]),
            "bf_bank_read": (i, [p, s, s, p]),
            "bf_bank_params": (i, [p, s, s, P(bf_chirp)]),
            "bf_opts_default": (None, [P(bf_opts)]),
            "bf_correlate": (i, [p, p, P(p), P(s), s, d, P(bf_opts), P(p)]),
            "bf_result_info_get": (i, [p, P(bf_result_info)]),
            "bf_result_check": (i, [p]),
            "bf_result_map_shape": (i, [p, s, P(s), P(s)]),
            "bf_result_get_max": (i, [p, s, P(p), P(p), P(p)]),
            "bf_result_get_hist": (i, [p, s, P(p)]),
            "bf_result_get_map": (i, [p, s, P(p)]),
            "bf_result_get_mean_max": (i, [p, P(p)]),
            "bf_result_copy_to_host": (i, [p, s, p, p, p, p, p]),
            "bf_result_copy_to_host_async": (i, [p, s, p, p, p, p, p, p]),
            "bf_result_copy_map_cells_async": (i, [p, s, p, p, s, p, p]),
            "bf_result_copy_mean_max": (i, [p, p]),
            "bf_result_fit_max": (i, [p, s, p, P(bf_skewnorm)]),
            "bf_result_coincidence": (i, [p, s, s, d, C.c_uint32, p, p, p, p, p]),
            "bf_result_tails": (i, [p, P(p), P(s)]),
            "bf_result_get_sigma_pred": (i, [p, s, P(p)]),
            "bf_result_copy_sigma_pred": (i, [p, s, p]),
            "bf_result_copy_tails": (i, [p, p, s, P(s)]),
            "bf_result_destroy": (None, [p]),
            "bf_plan_create": (i, [p, p, P(s), s, d, P(bf_opts), P(p)]),
            "bf_plan_run": (i, [p, P(p), p, P(p)]),
            "bf_plan_destroy": (None, [p]),
            "bf_control_randomize": (i, [p, p, s, u64, p]),
            "bf_control_randomize_static": (i, [p, s, u64, p, p]),
            "bf_serve_submit": (i, [p, P(bf_request), P(u64)]),
            "bf_serve_poll": (i, [p, u64, C.c_int64, P(p)]),
            "bf_serve_cancel": (i, [p, u64]),
            "bf_serve_stats_get": (i, [p, P(bf_serve_stats)]),
            "bf_last_error": (C.c_char_p, []),
            "bf_status_string": (C.c_char_p, [i]),
            "bf_abi_version": (i, []),
            "bf_selftest_wait": (i, [p, i, C.c_uint32, P(d)]),
            "bf_kernel_launches": (u64, []),
            "bf_probe_alu_peaks": (i, [i, P(d), P(d)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(st: int, ok=(BF_OK,)) -> int:
    if st not in ok:
        raise BFError(st, load().bf_last_error().decode())
    return st


def _addr(a) -> int:
    """Address of a numpy array or torch tensor (host or device)."""
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    if isinstance(a, np.ndarray):
        return int(a.ctypes.data)
    if isinstance(a, int):
        return a
    raise TypeError(type(a))


# ---------------------------------------------------------------- context
def bf_config_default() -> bf_config:
    c = bf_config()
    load().bf_config_default(C.byref(c))
    return c


def bf_init(cfg: bf_config | None = None) -> int:
    h = C.c_void_p()
    _check(load().bf_init(C.byref(cfg) if cfg is not None else None, C.byref(h)))
    return h.value


def bf_destroy(ctx: int) -> None:
    load().bf_destroy(ctx)


# ---------------------------------------------------------------- banks
def bf_bank_create(ctx: int, chirps, fs: float, T: float,
                   storage: int = BF_BANK_FP32 | BF_BANK_SPLIT_BF16) -> int:
    """chirps: sequence of (track, sense, f_lo, f_hi, sweep_s)."""
    arr = (bf_chirp * len(chirps))(*[bf_chirp(int(a), int(b), float(c), float(d), float(e))
                                     for a, b, c, d, e in chirps])
    h = C.c_void_p()
    _check(load().bf_bank_create(ctx, arr, len(chirps), fs, T, storage, C.byref(h)))
    return h.value


def bf_bank_create_grid(ctx: int, spec: dict, fs: float, T: float,
                        storage: int = BF_BANK_FP32 | BF_BANK_SPLIT_BF16) -> int:
    tr = (C.c_int32 * len(spec["tracks"]))(*spec["tracks"])
    se = (C.c_int32 * len(spec["senses"]))(*spec["senses"])
    du = (C.c_double * len(spec["durations"]))(*spec["durations"])
    g = bf_chirp_grid(tr, len(spec["tracks"]), se, len(spec["senses"]), du,
                      len(spec["durations"]), spec["f_min"], spec["f_max"], spec["I"], spec["J"])
    h = C.c_void_p()
    _check(load().bf_bank_create_grid(ctx, C.byref(g), fs, T, storage, C.byref(h)))
    return h.value


def bf_bank_destroy(bank: int) -> None:
    load().bf_bank_destroy(bank)


def bf_bank_size(bank: int) -> int:
    return int(load().bf_bank_size(bank))


def bf_bank_template_len(bank: int) -> int:
    return int(load().bf_bank_template_len(bank))


def bf_bank_rows(bank: int) -> int:
    return int(load().bf_bank_rows(bank))


def bf_bank_read(bank: int, k0: int, n: int) -> np.ndarray:
    """Templates [k0, k0+n); two rows per chirp (template, partner) for a
    quadrature bank."""
    M = bf_bank_template_len(bank)
    per = bf_bank_rows(bank) // bf_bank_size(bank)
    out = np.zeros((per * n, M), np.float32)
    _check(load().bf_bank_read(bank, k0, n, out.ctypes.data))
    return out


def bf_bank_params(bank: int, k0: int, n: int) -> list:
    arr = (bf_chirp * n)()
    _check(load().bf_bank_params(bank, k0, n, arr))
    return [(c.track, c.sense, c.f_lo, c.f_hi, c.sweep_s) for c in arr]


# ---------------------------------------------------------------- correlate
def bf_opts_default() -> bf_opts:
    o = bf_opts()
    load().bf_opts_default(C.byref(o))
    return o


def make_opts(precision=BF_SPLIT_BF16, bank_begin=0, bank_end=0, kappa=5.0, map_dt_s=1e-3,
              map_df_hz=4.0, want_map=False, want_hist=True, hist_bins=1024,
              stream=None, rho_out=None, want_tails=False, tile_lags=0,
              tail_sigma=BF_SIGMA_WHITE) -> bf_opts:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    o = bf_opts_default()
    o.precision = precision
    o.bank_begin = bank_begin
    o.bank_end = bank_end
    o.kappa = kappa
    o.map_dt_s = map_dt_s
    o.map_df_hz = map_df_hz
    o.want_map = int(bool(want_map))
    o.want_hist = int(bool(want_hist))
    o.hist_bins = hist_bins
    o.stream = stream
    o.rho_out = _addr(rho_out) if rho_out is not None else None
    o.want_tails = int(bool(want_tails))
    o.tile_lags = int(tile_lags)
    o.tail_sigma = int(tail_sigma)
    return o


def bf_correlate(ctx: int, bank: int, series, fs: float, opts: bf_opts | None = None,
                 lengths=None) -> int:
    """series: list of float32 arrays (numpy host arrays or torch tensors)."""
    n = len(series)
    ptrs = (C.c_void_p * n)(*[_addr(x) for x in series])
    if lengths is None:
        lengths = [x.numel() if hasattr(x, "numel") else len(x) for x in series]
    lens = (C.c_size_t * n)(*lengths)
    h = C.c_void_p()
    _check(load().bf_correlate(ctx, bank, ptrs, lens, n, fs,
                               C.byref(opts) if opts is not None else None, C.byref(h)))
    return h.value


def bf_result_check(res: int) -> None:
    """Raises BFError (BF_EINVAL) if a series of the finished result held a
    non-finite sample, (BF_EDEVICE) if a kernel reported a timed-out wait."""
    _check(load().bf_result_check(res))


def bf_result_info_get(res: int) -> bf_result_info:
    info = bf_result_info()
    _check(load().bf_result_info_get(res, C.byref(info)))
    return info


def bf_result_map_shape(res: int, s: int):
    nt, nf = C.c_size_t(), C.c_size_t()
    _check(load().bf_result_map_shape(res, s, C.byref(nt), C.byref(nf)))
    return nt.value, nf.value


def bf_result_get_max(res: int, s: int):
    a, b, c = C.c_void_p(), C.c_void_p(), C.c_void_p()
    _check(load().bf_result_get_max(res, s, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def bf_result_get_hist(res: int, s: int) -> int:
    a = C.c_void_p()
    _check(load().bf_result_get_hist(res, s, C.byref(a)))
    return a.value


def bf_result_get_map(res: int, s: int) -> int:
    a = C.c_void_p()
    _check(load().bf_result_get_map(res, s, C.byref(a)))
    return a.value


def bf_result_get_mean_max(res: int) -> int:
    a = C.c_void_p()
    _check(load().bf_result_get_mean_max(res, C.byref(a)))
    return a.value


def _copy_arrays(res: int, s: int, want_hist: bool, want_map: bool, out: dict | None) -> dict:
    """The host arrays a copy of series s writes: the caller's in ``out``,
    checked against the result's sizes and dtypes, else new ones."""
    info = bf_result_info_get(res)
    K = info.n_templates
    shapes = {"max": ((K,), np.float32), "argmax": ((K,), np.int32), "sigma": ((K,), np.float32)}
    if want_hist:
        shapes["hist"] = ((info.hist_bins,), np.uint32)
    if want_map:
        shapes["map"] = (tuple(bf_result_map_shape(res, s)), np.float32)
    arrs = {}
    for key, (shape, dt) in shapes.items():
        a = out.get(key) if out is not None else None
        if a is None:
            a = np.zeros(shape, dt)
        elif a.shape != shape or a.dtype != dt or not a.flags.c_contiguous or not a.flags.writeable:
            raise ValueError(f"out[{key!r}] must be a writeable C-contiguous {np.dtype(dt).name} "
                             f"array of shape {shape}")
        arrs[key] = a
    return dict(max=arrs["max"], argmax=arrs["argmax"], sigma=arrs["sigma"], hist=arrs.get("hist"),
                map=arrs.get("map"))


def _ptrs(a: dict):
    return [a[k].ctypes.data if a[k] is not None else None for k in ("max", "argmax", "sigma", "hist", "map")]


def bf_result_copy_to_host(res: int, s: int, want_hist=True, want_map=False, out: dict | None = None) -> dict:
    """Per-template max, argmax and sigma of series s, and optionally its
    histogram and map, copied into new numpy arrays, or into the caller's
    arrays in ``out`` (keys max, argmax, sigma, hist, map: C-contiguous, of the
    result's sizes and dtypes float32, int32, float32, uint32, float32), for
    instance views of pinned host memory reused across calls."""
    arrs = _copy_arrays(res, s, want_hist, want_map, out)
    _check(load().bf_result_copy_to_host(res, s, *_ptrs(arrs)))
    return arrs


def bf_result_copy_to_host_async(res: int, s: int, out: dict, stream=None, want_hist=True,
                                 want_map=False) -> dict:
    """Enqueues the copies of bf_result_copy_to_host into the caller's arrays
    ``out`` (page-locked host memory, e.g. numpy views of pinned torch
    tensors) on ``stream`` (a cudaStream_t handle such as
    ``torch.cuda.Stream().cuda_stream``; None: the legacy default stream) and
    returns at once. The arrays hold the outputs once the stream has been
    synchronised; ``res`` must not be destroyed before then."""
    arrs = _copy_arrays(res, s, want_hist, want_map, out)
    if any(out.get(k) is None for k, v in arrs.items() if v is not None):
        raise ValueError("an asynchronous copy needs every array it writes in `out`")
    _check(load().bf_result_copy_to_host_async(res, s, *_ptrs(arrs), stream))
    return arrs


def _addr(a) -> int:
    """Address of a torch tensor or a numpy array (no copy)."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def bf_result_copy_map_cells_async(res: int, s: int, cell, value, count, stream=None) -> None:
    """Enqueues the compaction of series s's painted map cells into ``cell``
    (uint32), ``value`` (float32), both of length cap, and ``count`` (one
    uint32): device tensors or page-locked host memory mapped into the
    device's address space (e.g. pinned torch tensors, or numpy views of
    them). After the stream is synchronised, count[0] is the number of
    painted cells and the first min(count[0], cap) entries hold them in
    increasing cell index."""
    cap = len(cell)
    if len(value) != cap or len(count) < 1:
        raise ValueError("cell and value must have the same length; count needs one element")
    _check(load().bf_result_copy_map_cells_async(res, s, _addr(cell) if cap else None,
                                                 _addr(value) if cap else None, cap, _addr(count), stream))


def bf_result_copy_mean_max(res: int) -> np.ndarray:
    K = bf_result_info_get(res).n_templates
    out = np.zeros(K, np.float32)
    _check(load().bf_result_copy_mean_max(res, out.ctypes.data))
    return out


def bf_result_fit_max(res: int, s: int = BF_FIT_MEAN, stream=None) -> dict:
    """Skew-normal fit of the maxima of series s (default: of their mean over
    series); returns the fields of bf_skewnorm as a dict."""
    out = bf_skewnorm()
    _check(load().bf_result_fit_max(res, s, stream, C.byref(out)))
    return {name: getattr(out, name) for name, _ in bf_skewnorm._fields_}


def bf_result_coincidence(res: int, a: int, b: int, delta_f_hz: float = 50.0, dt_cells: int = 0,
                          stream=None) -> dict:
    """Pseudo-spectra of tails of series a and b (independent and
    simultaneous counts per frequency cell of the map)."""
    nf = bf_result_map_shape(res, a)[1]
    out = {k: np.zeros(nf, np.uint32) for k in ("indep_a", "indep_b", "coinc_a", "coinc_b")}
    _check(load().bf_result_coincidence(res, a, b, float(delta_f_hz), int(dt_cells), stream,
                                        *[out[k].ctypes.data for k in ("indep_a", "indep_b",
                                                                        "coinc_a", "coinc_b")]))
    return out


TAIL_DTYPE = np.dtype([("series", np.uint32), ("k", np.uint32), ("tau", np.uint32),
                       ("rho", np.float32)])


def bf_result_tails(res: int):
    """(device address, count) of the kept tails."""
    a, n = C.c_void_p(), C.c_size_t()
    _check(load().bf_result_tails(res, C.byref(a), C.byref(n)))
    return a.value, n.value


def bf_result_copy_tails(res: int) -> np.ndarray:
    n = C.c_size_t()
    _check(load().bf_result_copy_tails(res, None, 0, C.byref(n)))
    out = np.zeros(n.value, TAIL_DTYPE)
    if n.value:
        _check(load().bf_result_copy_tails(res, out.ctypes.data, n.value, C.byref(n)))
    return out


def bf_result_get_sigma_pred(res: int, s: int) -> int:
    a = C.c_void_p()
    _check(load().bf_result_get_sigma_pred(res, s, C.byref(a)))
    return a.value


def bf_result_copy_sigma_pred(res: int, s: int) -> np.ndarray:
    out = np.zeros(bf_result_info_get(res).n_templates, np.float32)
    _check(load().bf_result_copy_sigma_pred(res, s, out.ctypes.data))
    return out


def bf_result_destroy(res: int) -> None:
    load().bf_result_destroy(res)


# ---------------------------------------------------------------- plans
def bf_plan_create(ctx: int, bank: int, lengths, fs: float, opts: bf_opts | None = None) -> int:
    n = len(lengths)
    lens = (C.c_size_t * n)(*lengths)
    h = C.c_void_p()
    _check(load().bf_plan_create(ctx, bank, lens, n, fs,
                                 C.byref(opts) if opts is not None else None, C.byref(h)))
    return h.value


def bf_plan_run(plan: int, series, stream=None) -> int:
    """Returns the plan's result handle (owned by the plan; do not destroy)."""
    n = len(series)
    ptrs = (C.c_void_p * n)(*[_addr(x) for x in series])
    h = C.c_void_p()
    _check(load().bf_plan_run(plan, ptrs, stream, C.byref(h)))
    return h.value


def bf_plan_destroy(plan: int) -> None:
    load().bf_plan_destroy(plan)


# ---------------------------------------------------------------- control
def bf_control_randomize(ctx: int, x, seed: int, out=None):
    """Returns out (a new float32 numpy array when out is None)."""
    n = x.numel() if hasattr(x, "numel") else len(x)
    if out is None:
        out = np.zeros(n, np.float32)
    _check(load().bf_control_randomize(ctx, _addr(x), n, seed & 0xFFFFFFFFFFFFFFFF, _addr(out)))
    return out


BF_STATIC_CONTROL_MAX = 524288


def bf_control_randomize_static(x, seed: int, out, stream=None) -> None:
    """Control without device allocation: x and out are CUDA tensors (or device
    addresses); enqueued on `stream` (a cudaStream_t handle, None = default)."""
    n = x.numel() if hasattr(x, "numel") else len(x)
    _check(load().bf_control_randomize_static(_addr(x), n, seed & 0xFFFFFFFFFFFFFFFF, _addr(out),
                                              stream))


# ---------------------------------------------------------------- serving
def bf_serve_submit(ctx: int, bank: int, series, fs: float, opts: bf_opts | None = None) -> int:
    n = series.numel() if hasattr(series, "numel") else len(series)
    req = bf_request(_addr(series), n, fs, bank, opts if opts is not None else bf_opts_default())
    t = C.c_uint64()
    _check(load().bf_serve_submit(ctx, C.byref(req), C.byref(t)))
    return t.value


def bf_serve_poll(ctx: int, ticket: int, timeout_us: int = -1):
    """Returns (status, result handle or None); BF_EPENDING / BF_ETIMEDOUT are
    returned, not raised."""
    h = C.c_void_p()
    st = _check(load().bf_serve_poll(ctx, ticket, timeout_us, C.byref(h)),
                ok=(BF_OK, BF_EPENDING, BF_ETIMEDOUT, BF_ECANCELED))
    return st, h.value


def bf_serve_cancel(ctx: int, ticket: int) -> None:
    _check(load().bf_serve_cancel(ctx, ticket))


def bf_serve_stats_get(ctx: int) -> bf_serve_stats:
    s = bf_serve_stats()
    _check(load().bf_serve_stats_get(ctx, C.byref(s)))
    return s


def bf_last_error() -> str:
    return load().bf_last_error().decode()


def bf_status_string(st: int) -> str:
    return load().bf_status_string(st).decode()


def bf_selftest_wait(ctx: int, signal: bool, limit_us: int) -> float:
    """Runs the bounded-wait self-test; returns the microseconds waited and
    raises BFError (BF_EDEVICE) when the wait ran out."""
    w = C.c_double()
    _check(load().bf_selftest_wait(ctx, int(bool(signal)), int(limit_us), C.byref(w)))
    return w.value


def bf_abi_version() -> int:
    return int(load().bf_abi_version())


def bf_kernel_launches() -> int:
    return int(load().bf_kernel_launches())


def bf_probe_alu_peaks(device: int = 0) -> tuple:
    """Measured FP32 and FP64 FMA rates of the device, TFLOP/s."""
    f32, f64 = C.c_double(), C.c_double()
    _check(load().bf_probe_alu_peaks(int(device), C.byref(f32), C.byref(f64)))
    return f32.value, f64.value
