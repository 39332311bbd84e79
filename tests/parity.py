"""Helpers shared by the GPU parity tests: run the CUDA library through the C
ABI and compare its outputs with the CPU oracle on the same seeded inputs."""
import numpy as np

import oracle
from paper_1802_01685_gb300 import bf

# per-result tolerances on normalised correlation (FP32, split-BF16 and the
# FP32 FFT route vs plain BF16 operands)
TOL = {"fp32": 2e-5, "split_bf16": 2e-5, "bf16": 1e-3, "fft_fp32": 2e-5, "split_fp16": 2e-5}

# every stored layout, so that one bank serves every route
STORE_ALL = bf.BF_BANK_FP32 | bf.BF_BANK_SPLIT_BF16 | bf.BF_BANK_SPLIT_FP16


def oracle_params(spec):
    return oracle.grid(spec["tracks"], spec["senses"], spec["durations"], spec["f_min"],
                       spec["f_max"], spec["I"], spec["J"])


def subset(params, idx):
    return {k: np.ascontiguousarray(v[idx]) for k, v in params.items()}


def top_two_margin(rho):
    """Per template: max |rho| minus the largest |rho| at any other lag."""
    a = np.abs(rho)
    top = a.argmax(axis=1)
    b = a.copy()
    b[np.arange(len(b)), top] = -1.0
    return a.max(axis=1) - b.max(axis=1)


def check_maxima(gpu, ref, rho_ref, tol, label=""):
    """max |rho| within tol per template; argmax equal wherever the oracle's
    top-two margin exceeds 2 tol.  Returns the fraction of argmaxes compared."""
    err = np.abs(gpu["max"].astype(np.float64) - ref["max"])
    assert err.max() <= tol, f"{label} max |rho| error {err.max():.3e} > {tol}"
    margin = top_two_margin(rho_ref)
    sel = margin > 2 * tol
    bad = np.nonzero(gpu["argmax"][sel] != ref["argmax"][sel])[0]
    assert len(bad) == 0, f"{label} argmax differs for {len(bad)} of {sel.sum()} templates"
    return float(sel.mean())


def check_sigma(gpu, ref, tol, label=""):
    err = np.abs(gpu["sigma"].astype(np.float64) - ref["sigma"])
    assert err.max() <= tol, f"{label} sigma error {err.max():.3e} > {tol}"


def check_hist(gpu_hist, ref_max, tol, nbins=1024):
    """Counts may differ only by maxima lying within tol of a bin edge."""
    ref = oracle.histogram(ref_max, nbins).astype(np.int64)
    g = gpu_hist.astype(np.int64)
    assert g.sum() == ref.sum() == len(ref_max)
    edges = np.arange(nbins + 1) / nbins
    near = np.zeros(nbins, np.int64)
    for v in ref_max:
        b = min(int(np.floor(v * nbins)), nbins - 1)
        if abs(v - edges[b]) <= tol or abs(edges[b + 1] - v) <= tol:
            near[max(b - 1, 0)] += 1
            near[b] += 1
            near[min(b + 1, nbins - 1)] += 1
    assert np.all(np.abs(g - ref) <= near), np.nonzero(np.abs(g - ref) > near)


def check_map(gpu_map, x, fs, params, M, kappa, tol, dt=1e-3, df=4.0):
    """Each GPU cell lies between the oracle maps painted at thr + tol and
    thr - tol, widened by tol."""
    thr = kappa / np.sqrt(M)
    hi = oracle.search(x, fs, params, M, thr=thr + tol, dt=dt, df=df, want_map=True)["map"]
    lo = oracle.search(x, fs, params, M, thr=thr - tol, dt=dt, df=df, want_map=True)["map"]
    assert gpu_map.shape == hi.shape
    g = gpu_map.astype(np.float64)
    assert np.all(g >= hi - tol), float((hi - tol - g).max())
    assert np.all(g <= lo + tol), float((g - lo - tol).max())
    return int((hi > 0).sum()), int((g > 0).sum())


def run(ctx, bank, series, fs, precision, **kw):
    res = bf.bf_correlate(ctx, bank, series, fs, bf.make_opts(precision=precision, **kw))
    try:
        info = bf.bf_result_info_get(res)
        outs = [bf.bf_result_copy_to_host(res, s, want_hist=kw.get("want_hist", True),
                                          want_map=kw.get("want_map", False))
                for s in range(len(series))]
        mean = bf.bf_result_copy_mean_max(res)
    finally:
        bf.bf_result_destroy(res)
    return outs, mean, info
