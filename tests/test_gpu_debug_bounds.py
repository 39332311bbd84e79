"""The debug build (libbf_debug.so, -DBF_DEBUG_BOUNDS): device-side bounds
checks that record a code in the context's status word instead of trapping,
and result buffers padded with canaries checked after every search.

The small parity cases of every route run on it in a fresh process: each
search must match the oracle and come back without BF_EDEVICE, i.e. no bounds
check fired and no output buffer was written past its end.  Then one canary
is overwritten on purpose (inside its allocation, so nothing faults) and
bf_result_check must report it."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCRIPT = textwrap.dedent("""
    import ctypes as C
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, "tests")
    import oracle
    from paper_1802_01685_gb300 import bf, synth
    from parity import STORE_ALL, TOL, check_hist, check_maxima, check_sigma, oracle_params, run, subset
    assert bf.LIB_PATH.endswith("libbf_debug.so"), bf.LIB_PATH
    ctx = bf.bf_init()
    w = synth.tiny(seed=1, n=6000, I=4, J=8)                  # 64 templates
    x, fs, M = w["series"][0], w["fs"], w["M"]
    p = oracle_params(w["grid"])
    ref = oracle.search(x, fs, p, M, want_rho=True)
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, M / fs, STORE_ALL)
    gen = bf.bf_bank_create_grid(ctx, w["grid"], fs, M / fs, bf.BF_BANK_GENERATED)
    for prec in ("split_bf16", "fp32", "bf16", "fft_fp32", "split_fp16"):
        for b in (bank, gen):
            outs, _, _ = run(ctx, b, [x, x[:4000].copy()], fs, prec, want_map=True, want_tails=True, kappa=3.0,
                             tail_sigma=bf.BF_SIGMA_PARSEVAL if prec == "fp32" else bf.BF_SIGMA_WHITE)
            check_maxima(outs[0], ref, ref["rho"], TOL[prec], prec)
            check_sigma(outs[0], ref, TOL[prec], prec)
            check_hist(outs[0]["hist"], ref["max"], TOL[prec])
        plan = bf.bf_plan_create(ctx, bank, [len(x)], fs, bf.make_opts(precision=prec, want_map=True))
        res = bf.bf_plan_run(plan, [x])
        bf.bf_result_check(res)
        bf.bf_plan_destroy(plan)
        t = bf.bf_serve_submit(ctx, bank, x, fs, bf.make_opts(precision=prec, bank_begin=3, bank_end=61))
        st, res = bf.bf_serve_poll(ctx, t, 60_000_000)
        assert st == bf.BF_OK
        bf.bf_result_check(res)
        bf.bf_result_destroy(res)
    # quadrature bank on the pair route of the FFT and the tensor cores
    chirps = [(bf.BF_LINEAR, bf.BF_ASC, 100.0, 700.0, 1.0), (bf.BF_POWERLAW, bf.BF_DESC, 40.0, 400.0, 0.6),
              (bf.BF_LINEAR, bf.BF_BOTH, 200.0, 600.0, 0.8)]
    qb = bf.bf_bank_create(ctx, chirps, fs, 1.0, STORE_ALL | bf.BF_BANK_QUADRATURE)
    for prec in ("split_bf16", "fft_fp32"):
        run(ctx, qb, [x], fs, prec, want_map=True, want_tails=True)
    bf.bf_bank_destroy(qb)
    # a canary overwritten on purpose: one byte past the end of vmax
    res = bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts())
    bf.bf_result_check(res)
    K = bf.bf_result_info_get(res).n_templates
    vmax = bf.bf_result_get_max(res, 0)[0]
    cudart = None
    for name in ("libcudart.so", "libcudart.so.13", "libcudart.so.12"):
        try:
            cudart = C.CDLL(name)
            break
        except OSError:
            pass
    assert cudart is not None, "no CUDA runtime library to write the canary with"
    cudart.cudaMemset.argtypes = [C.c_void_p, C.c_int, C.c_size_t]
    assert cudart.cudaMemset(C.c_void_p(vmax + 4 * K), 0, 1) == 0
    assert cudart.cudaDeviceSynchronize() == 0
    try:
        bf.bf_result_check(res)
        raise SystemExit("the overwritten canary was not reported")
    except bf.BFError as e:
        assert e.status == bf.BF_EDEVICE and "past its end" in str(e), str(e)
    bf.bf_result_destroy(res)
    bf.bf_bank_destroy(bank)
    bf.bf_bank_destroy(gen)
    bf.bf_destroy(ctx)
    print("debug build: every route clean, canary overwrite reported")
""")


def test_debug_build_checks_pass_and_canaries_detect_overruns():
    sys.path.insert(0, ROOT)
    from paper_1802_01685_gb300 import build as bfbuild
    import oracle
    lib = bfbuild.build(debug_bounds=True)
    oracle.build()
    env = dict(os.environ)
    env["BF_LIBRARY"] = lib
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", _SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "canary overwrite reported" in r.stdout
