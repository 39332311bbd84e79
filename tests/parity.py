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

# Bound on the L2 distance of a synthesised FP32 template row from the
# oracle's FP64 row.  By Cauchy-Schwarz a template off by dh moves rho by at
# most ||dh||_2 at any window, so this keeps the synthesis within a tenth of
# the 2e-5 budget on rho (the rows are unit-norm, Sect. 2.1 templates).
TEMPLATE_L2 = 2e-6


def bf16_rn(a):
    """FP32 values rounded to the nearest bfloat16 (ties to even), as FP32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split_decoded(h32, layout):
    """hi + lo of the tensor-core operand split of FP32 rows, as the bank read
    decodes it: BF16 hi = rn(h), lo = rn(h - hi); FP16 the same on 2^8 h."""
    h32 = np.asarray(h32, np.float32)
    if layout == "bf16":
        hi = bf16_rn(h32)
        return hi + bf16_rn(h32 - hi)
    hs = h32 * np.float32(256.0)
    hi = hs.astype(np.float16)
    lo = (hs - hi.astype(np.float32)).astype(np.float16)
    return hi.astype(np.float32) / np.float32(256.0) + lo.astype(np.float32) / np.float32(256.0)


def check_template_rows(h32, split, ref, label=""):
    """FP32 rows h32 within TEMPLATE_L2 (L2 norm) of the oracle rows ref;
    every split layout in `split` ({"bf16": rows, "fp16": rows}, hi + lo as
    read back) equal to the round-to-nearest split of h32 bit for bit, and
    within its own representation error (2^-16 relative for BF16 pairs,
    2^-22 for FP16 pairs) plus TEMPLATE_L2 of ref.  Returns the largest L2
    distance of the FP32 rows."""
    h32 = np.atleast_2d(np.asarray(h32, np.float32))
    ref = np.atleast_2d(np.asarray(ref, np.float64))
    d = np.sqrt(((h32.astype(np.float64) - ref) ** 2).sum(axis=1))
    assert d.max() <= TEMPLATE_L2, f"{label} template L2 error {d.max():.3e} > {TEMPLATE_L2}"
    for layout, rows in split.items():
        rows = np.atleast_2d(np.asarray(rows, np.float32))
        want = split_decoded(h32, layout)
        assert np.array_equal(rows, want), f"{label} {layout} split differs from rn split of the FP32 row"
        rel = 2.0 ** -16 if layout == "bf16" else 2.0 ** -22
        rep = np.sqrt(((rows.astype(np.float64) - h32) ** 2).sum(axis=1))
        n32 = np.sqrt((h32.astype(np.float64) ** 2).sum(axis=1))
        assert np.all(rep <= rel * n32), f"{label} {layout} split error above {rel:.1e} relative"
        dd = np.sqrt(((rows.astype(np.float64) - ref) ** 2).sum(axis=1))
        assert np.all(dd <= rep + TEMPLATE_L2), f"{label} {layout} rows off the oracle"
    return float(d.max())


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
