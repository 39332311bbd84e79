"""Randomised parity: seeded draws of template length (odd lengths and
lengths off the 64-sample grid included), sample rate, chirp mix (tracks,
senses, sweep times), quadrature or not, series lengths down to N = M, bank
slices and route, each compared with the oracle on the dense output and the
maxima.  Each case is small enough for the oracle to finish in a second."""
import os

import numpy as np
import pytest

import oracle
from paper_1802_01685_gb300 import bf

from parity import STORE_ALL, TOL, check_maxima

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROUTES = ["split_bf16", "fp32", "bf16", "fft_fp32", "split_fp16"]


def seeds(start, n):
    """The seeds of a family of draws: n of them, or n times BF_RANDOM_REPEAT
    for a longer soak (the first n are always the same)."""
    return range(start, start + n * max(1, int(os.environ.get("BF_RANDOM_REPEAT", "1"))))


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    h = bf.bf_init()
    yield h
    bf.bf_destroy(h)


def draw_case(seed):
    r = np.random.default_rng(seed)
    M = int(r.choice([97, 250, 512, 777, 1000, 1024, 1500, 2000, 2048, 3001, 4096]))
    T = 1.0
    fs = float(M) / T
    K = int(r.integers(3, 40))
    chirps = []
    for _ in range(K):
        track = int(r.integers(2))
        sense = int(r.integers(3))
        f_lo = float(r.uniform(0.01, 0.2) * fs)
        f_hi = float(min(f_lo * r.uniform(1.2, 6.0), 0.45 * fs))
        D = float(r.uniform(max(2.0 / fs, 0.15), 1.0))
        chirps.append((track, sense, f_lo, f_hi, D))
    quad = bool(r.integers(4) == 0)
    n_series = int(r.integers(1, 4))
    lens = [M + int(r.choice([0, 1, int(r.integers(2, 2 * M))])) for _ in range(n_series)]
    b0 = int(r.integers(0, K // 3 + 1))
    b1 = int(r.integers(max(b0 + 1, 2 * K // 3), K + 1))
    route = ROUTES[seed % len(ROUTES)]
    return dict(M=M, fs=fs, chirps=chirps, quad=quad, lens=lens, b0=b0, b1=b1, route=route, rng=r)


@pytest.mark.parametrize("seed", seeds(0, 200))
def test_random_case(ctx, seed):
    c = draw_case(seed)
    fs, M, route = c["fs"], c["M"], c["route"]
    if route == "fft_fp32" and M > 4096:
        pytest.skip("FFT route: templates of at most 4096 samples")
    r = c["rng"]
    xs = []
    for n in c["lens"]:
        x = r.standard_normal(n)
        if r.integers(2):                               # a bank template placed in the noise
            k = int(r.integers(len(c["chirps"])))
            h = oracle.template(*c["chirps"][k], fs, M, 0)
            o = int(r.integers(0, n - M + 1))
            x[o:o + M] += float(r.uniform(2.0, 20.0)) * h
        xs.append(x.astype(np.float32))
    storage = STORE_ALL | (bf.BF_BANK_QUADRATURE if c["quad"] else 0)
    bank = bf.bf_bank_create(ctx, c["chirps"], fs, 1.0, storage)
    p = {k: np.array([ch[i] for ch in c["chirps"][c["b0"]:c["b1"]]], dt)
         for i, (k, dt) in enumerate((("track", np.int32), ("sense", np.int32), ("f_lo", np.float64),
                                      ("f_hi", np.float64), ("D", np.float64)))}
    tol = TOL[route]
    if route == "bf16" and M < 1024:
        # plain BF16 rounds each operand to 2^-9: by Cauchy-Schwarz |drho| <= 2^-8 at
        # any M; the stated 1e-3 relies on the averaging of long templates
        tol = 2.0 ** -8
    res = bf.bf_correlate(ctx, bank, xs, fs, bf.make_opts(precision=route, bank_begin=c["b0"], bank_end=c["b1"]))
    outs = [bf.bf_result_copy_to_host(res, s) for s in range(len(xs))]
    bf.bf_result_destroy(res)
    for s, x in enumerate(xs):
        ref = oracle.search(x, fs, p, M, want_rho=True, quadrature=c["quad"])
        check_maxima(outs[s], ref, ref["rho"], tol, f"seed {seed} series {s} ({route}, M={M})")
        if s == 0:
            K, L = ref["rho"].shape
            rho = torch.zeros((K, L), dtype=torch.float32, device="cuda")
            bf.bf_result_destroy(bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts(
                precision=route, bank_begin=c["b0"], bank_end=c["b1"], rho_out=rho)))
            err = np.abs(rho.cpu().numpy().astype(np.float64) - ref["rho"]).max()
            assert err <= tol, (seed, route, M, err)
    bf.bf_bank_destroy(bank)


@pytest.mark.parametrize("seed", seeds(0, 60))
def test_random_case_generated_bank_and_plan(ctx, seed):
    """The same draws through a generated bank and through a captured plan:
    maxima, argmaxes and sigma bit for bit equal to bf_correlate with the
    stored bank (the plan with white tails; sigma to rounding, its sums are
    atomics)."""
    c = draw_case(seed)
    fs, M, route = c["fs"], c["M"], c["route"]
    if route == "fft_fp32" and M > 4096:
        pytest.skip("FFT route: templates of at most 4096 samples")
    r = c["rng"]
    xs = [r.standard_normal(n).astype(np.float32) for n in c["lens"]]
    q = bf.BF_BANK_QUADRATURE if c["quad"] else 0
    stored = bf.bf_bank_create(ctx, c["chirps"], fs, 1.0, STORE_ALL | q)
    gen = bf.bf_bank_create(ctx, c["chirps"], fs, 1.0, bf.BF_BANK_GENERATED | q)
    opts = bf.make_opts(precision=route, bank_begin=c["b0"], bank_end=c["b1"])

    def outs(res, owned=True):
        o = [bf.bf_result_copy_to_host(res, s) for s in range(len(xs))]
        if owned:
            bf.bf_result_destroy(res)
        return o

    ref = outs(bf.bf_correlate(ctx, stored, xs, fs, opts))
    g = outs(bf.bf_correlate(ctx, gen, xs, fs, opts))
    plan = bf.bf_plan_create(ctx, stored, c["lens"], fs, opts)
    pl = outs(bf.bf_plan_run(plan, xs), owned=False)          # the plan owns its result
    for s in range(len(xs)):
        for other in (g[s], pl[s]):
            np.testing.assert_array_equal(other["max"], ref[s]["max"])
            np.testing.assert_array_equal(other["argmax"], ref[s]["argmax"])
            np.testing.assert_allclose(other["sigma"], ref[s]["sigma"], rtol=1e-6, atol=1e-12)
    bf.bf_plan_destroy(plan)
    bf.bf_bank_destroy(stored)
    bf.bf_bank_destroy(gen)


@pytest.mark.parametrize("seed", list(seeds(300, 40)) + [500, 1345, 1988, 2057, 2167])
def test_random_case_tails_and_map(ctx, seed):
    """Tails |rho| >= kappa sigma_white and the time-frequency map they paint,
    for random draws, against the oracle at the same threshold: every tail
    the oracle finds above thr + tol is listed, none below thr - tol, and
    every map cell lies between the oracle maps painted at thr -/+ tol.
    Seeds 500, 1345, 1988, 2057 and 2167 draw M = fs = 2000 with sweeps
    ending at f_hi = 900 Hz, a 4 Hz cell edge, where the clamped end of the
    track once fell on either side of the edge."""
    c = draw_case(seed)
    fs, M, route = c["fs"], c["M"], c["route"]
    if route == "fft_fp32" and M > 4096:
        pytest.skip("FFT route: templates of at most 4096 samples")
    r = c["rng"]
    x = r.standard_normal(c["lens"][0] + M)
    k = int(r.integers(c["b0"], c["b1"]))
    x[M // 2:M // 2 + M] += 6.0 * oracle.template(*c["chirps"][k], fs, M, 0)
    x = x.astype(np.float32)
    q = bf.BF_BANK_QUADRATURE if c["quad"] else 0
    bank = bf.bf_bank_create(ctx, c["chirps"], fs, 1.0, STORE_ALL | q)
    p = {kk: np.array([ch[i] for ch in c["chirps"][c["b0"]:c["b1"]]], dt)
         for i, (kk, dt) in enumerate((("track", np.int32), ("sense", np.int32), ("f_lo", np.float64),
                                       ("f_hi", np.float64), ("D", np.float64)))}
    tol = TOL[route] if not (route == "bf16" and M < 1024) else 2.0 ** -8
    kappa = 3.0
    thr = kappa * np.sqrt((2.0 if c["quad"] else 1.0) / M)
    res = bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts(precision=route, bank_begin=c["b0"],
                                                           bank_end=c["b1"], kappa=kappa,
                                                           want_tails=True, want_map=True))
    tails = bf.bf_result_copy_tails(res)
    mp = bf.bf_result_copy_to_host(res, 0, want_map=True)["map"]
    bf.bf_result_destroy(res)
    ref = oracle.search(x, fs, p, M, want_rho=True, quadrature=c["quad"])
    a = np.abs(ref["rho"])
    koff = c["b0"]
    got = {(int(t["k"]) - koff, int(t["tau"])) for t in tails}
    must = set(zip(*[v.tolist() for v in np.nonzero(a >= thr + tol)]))
    may = set(zip(*[v.tolist() for v in np.nonzero(a >= thr - tol)]))
    assert must <= got <= may, (seed, route, len(must - got), len(got - may))
    hi = oracle.search(x, fs, p, M, thr=thr + tol, want_map=True, quadrature=c["quad"])["map"]
    lo = oracle.search(x, fs, p, M, thr=thr - tol, want_map=True, quadrature=c["quad"])["map"]
    assert mp.shape == hi.shape
    assert np.all(mp >= hi - tol) and np.all(mp <= lo + tol), (seed, route)
    bf.bf_bank_destroy(bank)


@pytest.mark.parametrize("seed", seeds(500, 1))
def test_random_serving_mix(ctx, seed):
    """Thirty random requests (lengths, bank slices, routes, map and tails on or
    off) against a plain and a quadrature bank, all submitted at once: each
    result equals, bit for bit, the same search run alone."""
    rng = np.random.default_rng(seed)
    fs = 2048.0
    chirps = []
    for _ in range(300):
        f_lo = float(rng.uniform(20.0, 300.0))
        chirps.append((int(rng.integers(2)), int(rng.integers(3)), f_lo,
                       float(min(f_lo * rng.uniform(1.3, 5.0), 950.0)), float(rng.uniform(0.3, 1.0))))
    banks = [bf.bf_bank_create(ctx, chirps, fs, 1.0, STORE_ALL),
             bf.bf_bank_create(ctx, chirps, fs, 1.0, STORE_ALL | bf.BF_BANK_QUADRATURE)]
    reqs = []
    for i in range(30):
        n = int(rng.integers(2048, 40000))
        b0 = int(rng.integers(0, 150))
        b1 = int(rng.integers(b0 + 1, 301))
        route = ROUTES[int(rng.integers(len(ROUTES)))]
        x = rng.standard_normal(n).astype(np.float32)
        opts = bf.make_opts(precision=route, bank_begin=b0, bank_end=b1, want_map=bool(rng.integers(2)),
                            want_tails=bool(rng.integers(2)), kappa=4.0)
        reqs.append((banks[int(rng.integers(2))], x, opts))

    def fetch(res, opts):
        o = bf.bf_result_copy_to_host(res, 0, want_hist=True, want_map=bool(opts.want_map))
        if opts.want_tails:
            o["tails"] = np.sort(bf.bf_result_copy_tails(res), order=["k", "tau"])
        bf.bf_result_destroy(res)
        return o

    alone = [fetch(bf.bf_correlate(ctx, b, [x], fs, o), o) for b, x, o in reqs]
    tickets = [bf.bf_serve_submit(ctx, b, x, fs, o) for b, x, o in reqs]
    for t, (b, x, o), a in zip(tickets, reqs, alone):
        st, res = bf.bf_serve_poll(ctx, t, 120_000_000)
        assert st == bf.BF_OK
        m = fetch(res, o)
        np.testing.assert_array_equal(m["max"], a["max"])
        np.testing.assert_array_equal(m["argmax"], a["argmax"])
        np.testing.assert_allclose(m["sigma"], a["sigma"], rtol=1e-6, atol=1e-12)
        np.testing.assert_array_equal(m["hist"], a["hist"])
        if o.want_map:
            np.testing.assert_array_equal(m["map"], a["map"])
        if o.want_tails:
            np.testing.assert_array_equal(m["tails"], a["tails"])
    for b in banks:
        bf.bf_bank_destroy(b)


@pytest.mark.parametrize("route", ROUTES)
def test_more_series_than_one_launch_holds(ctx, route):
    """130 series of random lengths in one call: more than a launch holds (64
    segments or 64 FFT series), so the call splits into several launches.
    Every series' maxima and the mean over series match the oracle."""
    rng = np.random.default_rng(600 + ROUTES.index(route))
    fs, M = 256.0, 256
    chirps = [(int(rng.integers(2)), int(rng.integers(3)), float(f), float(f * rng.uniform(1.5, 3.0)),
               float(rng.uniform(0.4, 1.0))) for f in rng.uniform(5.0, 40.0, 20)]
    bank = bf.bf_bank_create(ctx, chirps, fs, 1.0, STORE_ALL)
    p = {k: np.array([ch[i] for ch in chirps], dt)
         for i, (k, dt) in enumerate((("track", np.int32), ("sense", np.int32), ("f_lo", np.float64),
                                      ("f_hi", np.float64), ("D", np.float64)))}
    xs = [rng.standard_normal(int(rng.integers(M, 4 * M))).astype(np.float32) for _ in range(130)]
    outs, mean, info = [None], None, None
    res = bf.bf_correlate(ctx, bank, xs, fs, bf.make_opts(precision=route))
    outs = [bf.bf_result_copy_to_host(res, s) for s in range(len(xs))]
    mean = bf.bf_result_copy_mean_max(res)
    bf.bf_result_destroy(res)
    tol = TOL[route] if route != "bf16" else 2.0 ** -8
    acc = np.zeros(len(chirps))
    for s, x in enumerate(xs):
        ref = oracle.search(x, fs, p, M, want_rho=True)
        check_maxima(outs[s], ref, ref["rho"], tol, f"{route} series {s}")
        acc += ref["max"]
    np.testing.assert_allclose(mean, acc / len(xs), atol=tol)


@pytest.mark.parametrize("seed", seeds(700, 12))
def test_random_parseval_predictor(ctx, seed):
    """The Parseval-predicted sigma of random banks and series (white, red and
    Poisson-like) against the oracle's."""
    c = draw_case(seed)
    fs, M = c["fs"], c["M"]
    r = c["rng"]
    n = c["lens"][0] + 2 * M
    kind = seed % 3
    x = r.standard_normal(n)
    if kind == 1:
        x = np.cumsum(x) * 0.05 + x                    # red
    elif kind == 2:
        x = r.poisson(3.0, n) - 3.0                     # counts, mean removed
    x = x.astype(np.float32)
    bank = bf.bf_bank_create(ctx, c["chirps"], fs, 1.0, STORE_ALL)
    res = bf.bf_correlate(ctx, bank, [x], fs, bf.make_opts(precision="split_bf16", bank_begin=c["b0"],
                                                           bank_end=c["b1"], tail_sigma=bf.BF_SIGMA_PARSEVAL))
    got = bf.bf_result_copy_sigma_pred(res, 0).astype(np.float64)
    bf.bf_result_destroy(res)
    p = {k: np.array([ch[i] for ch in c["chirps"][c["b0"]:c["b1"]]], dt)
         for i, (k, dt) in enumerate((("track", np.int32), ("sense", np.int32), ("f_lo", np.float64),
                                      ("f_hi", np.float64), ("D", np.float64)))}
    ref = oracle.parseval_sigma(x, oracle.bank(p, fs, M))
    np.testing.assert_allclose(got, ref, rtol=2e-5, atol=1e-9)
    bf.bf_bank_destroy(bank)
