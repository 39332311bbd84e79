"""Serving with continuous batching, through the C ABI."""
import time

import numpy as np
import pytest

import oracle
from paper_1802_01685_gb300 import bf, synth

from parity import TOL, check_hist, check_map, check_maxima, check_sigma, oracle_params, subset

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FS, T = 2048.0, 1.0


@pytest.fixture(scope="module")
def served():
    import __graft_entry__
    __graft_entry__.build()
    cfg = bf.bf_config_default()
    cfg.serve_slots = 4
    ctx = bf.bf_init(cfg)
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0, 0.5],
                           20.0, 1000.0, 16, 16)                 # 2048 templates
    bank = bf.bf_bank_create_grid(ctx, spec, FS, T,
                                  bf.BF_BANK_FP32 | bf.BF_BANK_SPLIT_BF16 | bf.BF_BANK_SPLIT_FP16)
    yield ctx, bank, spec
    bf.bf_bank_destroy(bank)
    bf.bf_destroy(ctx)


PREC = {bf.BF_SPLIT_BF16: "split_bf16", bf.BF_BF16: "bf16", bf.BF_FP32: "fp32",
        bf.BF_FFT_FP32: "fft_fp32", bf.BF_SPLIT_FP16: "split_fp16"}


def requests():
    rng = np.random.default_rng(21)
    out = []
    for i, (secs, k0, k1, prec, mp) in enumerate([
            (3.0, 0, 2048, "split_bf16", False), (7.5, 100, 1900, "split_bf16", True),
            (2.0, 0, 512, "bf16", False), (12.25, 640, 2048, "split_bf16", False),
            (4.0, 0, 1024, "fp32", True), (1.0 + 1 / 2048, 5, 133, "split_bf16", False),
            (5.0, 64, 1500, "split_bf16", True), (3.5, 0, 2048, "split_bf16", False),
            (6.0, 17, 2000, "fft_fp32", True), (9.0, 0, 2048, "fft_fp32", False),
            (4.5, 30, 1800, "split_fp16", True), (2.5, 0, 2048, "split_fp16", False)]):
        n = int(secs * FS)
        x = synth.white(n, rng).astype(np.float32) if i % 2 == 0 else \
            synth.grb_lightcurve(n, FS, rng).astype(np.float32)
        out.append((x, bf.make_opts(precision=prec, bank_begin=k0, bank_end=k1, want_map=mp,
                                    kappa=4.0, want_tails=mp or i == 7,
                                    tail_sigma=bf.BF_SIGMA_PARSEVAL if i == 6 else bf.BF_SIGMA_WHITE)))
    return out


def fetch(res, want_map, parseval=False, tails=False):
    r = bf.bf_result_copy_to_host(res, 0, want_hist=True, want_map=want_map)
    if parseval:
        r["sigma_pred"] = bf.bf_result_copy_sigma_pred(res, 0)
    if tails:
        r["tails"] = np.sort(bf.bf_result_copy_tails(res), order=["k", "tau"])
    bf.bf_result_destroy(res)
    return r


def test_each_result_is_the_same_alone_and_in_the_mix(served):
    """Twelve requests of every route, bank slice, length and series kind
    submitted together: each served result equals the oracle within its
    route's tolerance, and the same search run alone bit for bit."""
    ctx, bank, spec = served
    params = oracle_params(spec)
    reqs = requests()
    alone = [fetch(bf.bf_correlate(ctx, bank, [x], FS, o), o.want_map, o.tail_sigma == 1,
                   o.want_tails == 1) for x, o in reqs]
    tickets = [bf.bf_serve_submit(ctx, bank, x, FS, o) for x, o in reqs]
    mixed = []
    for t, (x, o) in zip(tickets, reqs):
        st, res = bf.bf_serve_poll(ctx, t, 60_000_000)
        assert st == bf.BF_OK
        mixed.append(fetch(res, o.want_map, o.tail_sigma == 1, o.want_tails == 1))
    for (x, o), m in zip(reqs, mixed):
        # the served result itself against the oracle on the same inputs
        tol = TOL[PREC[o.precision]]
        k0, k1 = o.bank_begin, o.bank_end
        p = subset(params, np.arange(k0, k1))
        ref = oracle.search(x, FS, p, int(FS), want_rho=True)
        check_maxima(m, ref, ref["rho"], tol, f"served {PREC[o.precision]} [{k0}, {k1})")
        check_sigma(m, ref, tol, "served")
        check_hist(m["hist"], ref["max"], tol)
        if o.want_map and o.tail_sigma != bf.BF_SIGMA_PARSEVAL:       # maps painted at kappa / sqrt(M)
            check_map(m["map"], x, FS, p, int(FS), o.kappa, tol)
    for a, m in zip(alone, mixed):
        np.testing.assert_array_equal(m["max"], a["max"])
        np.testing.assert_array_equal(m["argmax"], a["argmax"])
        np.testing.assert_allclose(m["sigma"], a["sigma"], rtol=1e-6, atol=1e-9)
        np.testing.assert_array_equal(m["hist"], a["hist"])
        if a["map"] is not None:
            np.testing.assert_array_equal(m["map"], a["map"])
        if "sigma_pred" in a:
            np.testing.assert_array_equal(m["sigma_pred"], a["sigma_pred"])
        if "tails" in a:
            assert len(a["tails"]) > 0
            np.testing.assert_array_equal(m["tails"], a["tails"])
    s = bf.bf_serve_stats_get(ctx)
    assert s.completed >= len(reqs) and s.p99_ms >= s.p50_ms > 0


def test_late_small_request_joins_and_finishes_first(served):
    ctx, bank, _ = served
    rng = np.random.default_rng(5)
    big = synth.white(int(600 * FS), rng).astype(np.float32)     # 10 minutes x 2048 templates, FP32
    small = synth.white(int(2 * FS), rng).astype(np.float32)
    o_big = bf.make_opts(precision="fp32")
    o_small = bf.make_opts(precision="split_bf16", bank_end=256)
    tb = bf.bf_serve_submit(ctx, bank, big, FS, o_big)
    for _ in range(2000):                                        # wait until the big one runs
        if bf.bf_serve_stats_get(ctx).active >= 1:
            break
        time.sleep(0.001)
    ts = bf.bf_serve_submit(ctx, bank, small, FS, o_small)
    st, rs = bf.bf_serve_poll(ctx, ts, 60_000_000)
    assert st == bf.BF_OK
    st_big, rb = bf.bf_serve_poll(ctx, tb, 0)
    assert st_big == bf.BF_EPENDING, "small request waited for the big one"
    st_big, rb = bf.bf_serve_poll(ctx, tb, 120_000_000)
    assert st_big == bf.BF_OK
    ref = fetch(bf.bf_correlate(ctx, bank, [small], FS, o_small), False)
    np.testing.assert_array_equal(fetch(rs, False)["max"], ref["max"])
    bf.bf_result_destroy(rb)


def test_cancel_and_unknown_ticket(served):
    ctx, bank, _ = served
    x = synth.white(int(200 * FS), np.random.default_rng(1)).astype(np.float32)
    t = bf.bf_serve_submit(ctx, bank, x, FS, bf.make_opts(precision="fp32"))
    bf.bf_serve_cancel(ctx, t)
    st, res = bf.bf_serve_poll(ctx, t, 60_000_000)
    assert st == bf.BF_ECANCELED and res is None
    with pytest.raises(bf.BFError) as e:
        bf.bf_serve_poll(ctx, t, 0)                              # ticket is gone
    assert e.value.status == bf.BF_EINVAL


def test_queue_full_and_budget():
    import __graft_entry__
    __graft_entry__.build()
    cfg = bf.bf_config_default()
    cfg.serve_slots = 1
    cfg.serve_queue = 1
    ctx = bf.bf_init(cfg)
    spec = synth.grid_spec([synth.LINEAR], [synth.ASC], [1.0], 20.0, 1000.0, 16, 16)
    bank = bf.bf_bank_create_grid(ctx, spec, FS, T)
    x = synth.white(int(120 * FS), np.random.default_rng(2)).astype(np.float32)
    opts = bf.make_opts(precision="fp32")
    tickets, again = [], False
    for _ in range(50):
        try:
            tickets.append(bf.bf_serve_submit(ctx, bank, x, FS, opts))
        except bf.BFError as e:
            assert e.status == bf.BF_EAGAIN
            again = True
            break
    assert again
    for t in tickets:
        bf.bf_serve_cancel(ctx, t)
        bf.bf_serve_poll(ctx, t, 120_000_000)
    bf.bf_bank_destroy(bank)
    bf.bf_destroy(ctx)

    cfg = bf.bf_config_default()
    cfg.hbm_budget = 64 << 20
    ctx = bf.bf_init(cfg)
    bank = bf.bf_bank_create_grid(ctx, spec, FS, T)              # 256 x 2048: fits
    huge = np.zeros(int(1200 * FS), np.float32)
    with pytest.raises(bf.BFError) as e:
        bf.bf_serve_submit(ctx, bank, huge, FS, bf.make_opts(precision="split_bf16"))
    assert e.value.status == bf.BF_ENOMEM
    with pytest.raises(bf.BFError) as e:
        bf.bf_bank_create_grid(ctx, synth.grid_spec([0], [0], [1.0], 20.0, 1000.0, 128, 128), FS, T)
    assert e.value.status == bf.BF_ENOMEM
    bf.bf_bank_destroy(bank)
    bf.bf_destroy(ctx)


def test_shortest_policy_same_results_and_small_requests_first():
    """BF_SERVE_SHORTEST changes only the order of the work: the twelve-request
    mix gives, request by request, what the same searches alone give, bit for
    bit; and with one slot, a small request queued behind a large one is
    admitted first (the large one is still pending when the small one is
    done)."""
    import __graft_entry__
    __graft_entry__.build()
    cfg = bf.bf_config_default()
    cfg.serve_slots = 4
    cfg.serve_policy = bf.BF_SERVE_SHORTEST
    ctx = bf.bf_init(cfg)
    spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0, 0.5],
                           20.0, 1000.0, 16, 16)                 # 2048 templates
    bank = bf.bf_bank_create_grid(ctx, spec, FS, T,
                                  bf.BF_BANK_FP32 | bf.BF_BANK_SPLIT_BF16 | bf.BF_BANK_SPLIT_FP16)
    try:
        reqs = requests()
        alone = [fetch(bf.bf_correlate(ctx, bank, [x], FS, o), o.want_map) for x, o in reqs]
        tickets = [bf.bf_serve_submit(ctx, bank, x, FS, o) for x, o in reqs]
        for t, (x, o), a in zip(tickets, reqs, alone):
            st, res = bf.bf_serve_poll(ctx, t, 60_000_000)
            assert st == bf.BF_OK
            m = fetch(res, o.want_map)
            np.testing.assert_array_equal(m["max"], a["max"])
            np.testing.assert_array_equal(m["argmax"], a["argmax"])
            np.testing.assert_array_equal(m["hist"], a["hist"])
            if a["map"] is not None:
                np.testing.assert_array_equal(m["map"], a["map"])
    finally:
        bf.bf_bank_destroy(bank)
        bf.bf_destroy(ctx)

    cfg.serve_slots = 1
    ctx = bf.bf_init(cfg)
    bank = bf.bf_bank_create_grid(ctx, spec, FS, T)
    try:
        rng = np.random.default_rng(9)
        big = [synth.white(int(600 * FS), rng).astype(np.float32) for _ in range(2)]
        small = synth.white(int(2 * FS), rng).astype(np.float32)
        o_big = bf.make_opts(precision="fp32")
        o_small = bf.make_opts(precision="split_bf16", bank_end=256)
        t1 = bf.bf_serve_submit(ctx, bank, big[0], FS, o_big)
        for _ in range(2000):                                    # the first one runs
            if bf.bf_serve_stats_get(ctx).active >= 1:
                break
            time.sleep(0.001)
        t2 = bf.bf_serve_submit(ctx, bank, big[1], FS, o_big)
        ts = bf.bf_serve_submit(ctx, bank, small, FS, o_small)
        st, rs = bf.bf_serve_poll(ctx, ts, 120_000_000)
        assert st == bf.BF_OK
        assert bf.bf_serve_poll(ctx, t2, 0)[0] == bf.BF_EPENDING, "the large request was admitted first"
        ref = fetch(bf.bf_correlate(ctx, bank, [small], FS, o_small), False)
        np.testing.assert_array_equal(fetch(rs, False)["max"], ref["max"])
        for t in (t1, t2):
            st, r = bf.bf_serve_poll(ctx, t, 240_000_000)
            assert st == bf.BF_OK
            bf.bf_result_destroy(r)
    finally:
        bf.bf_bank_destroy(bank)
        bf.bf_destroy(ctx)
