"""Serving loop: continuous batching with resident plans and pattern tables.

Every request's result must be the same bits alone and in the mix (the
arithmetic is exact, so the tolerance is zero), and agree with the oracle on
the request's own input.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_0907_1788_gb300 import build

    build.build()
    import paper_0907_1788_gb300 as pkg

    pkg.load()
    oracle.build()
    return pkg


def _trace(n_req=48):
    reqs = synth.serving_requests(seed=9, rate_per_s=2000.0, duration_s=1.0, log2n=(6, 14),
                                  log2bytes=(7, 10), patterns_per_shape=3)[:n_req]
    out = []
    for q in reqs:
        d = dict(op=q["op"], n=q["n"], k=q["k"], W=q["W"], seed=q["seed"], t=q["t"])
        if q["op"] == "decode":
            d["positions"] = synth.received_positions(
                q["n"], synth.erased_uniform(q["pattern_seed"], q["n"], q["k"]))
        out.append(d)
    return out


def _run(pkg, reqs, nstreams, one_by_one):
    srv = pkg.fnt_rs_server_create(1 << 30, nstreams=nstreams, keep_results=True)
    try:
        results = []
        tickets = []
        for q in reqs:
            t = pkg.fnt_rs_server_submit(srv, q)
            tickets.append(t)
            if one_by_one:
                pkg.fnt_rs_server_drain(srv)
        pkg.fnt_rs_server_drain(srv)
        for q, t in zip(reqs, tickets):
            done, lat = pkg.fnt_rs_server_poll(srv, t)
            assert done and lat >= 0
            results.append(pkg.fnt_rs_server_fetch(srv, t, q))
            pkg.fnt_rs_server_release(srv, t)
        return results
    finally:
        pkg.fnt_rs_server_destroy(srv)


def test_same_alone_and_in_mix_and_oracle(pkg):
    reqs = _trace()
    assert {q["op"] for q in reqs} == {"encode", "decode"}
    mix = _run(pkg, reqs, nstreams=8, one_by_one=False)
    alone = _run(pkg, reqs, nstreams=1, one_by_one=True)
    for q, (a_in, a_out), (b_in, b_out) in zip(reqs, alone, mix):
        assert np.array_equal(a_in, b_in) and np.array_equal(a_out, b_out), q
    for q, (h_in, h_out) in list(zip(reqs, mix))[:16]:
        if q["op"] == "encode":
            assert np.array_equal(h_out, oracle.encode(h_in, q["n"]))
        else:
            want, _ = oracle.decode(h_in, q["positions"][: q["k"]], q["n"], q["k"])
            assert np.array_equal(h_out, want)


def test_budget_and_replay(pkg):
    srv = pkg.fnt_rs_server_create(8 << 20, nstreams=4, keep_results=False)
    try:  # buffers alone larger than the arena: refused at submit
        with pytest.raises(pkg.FntRsError) as ei:
            pkg.fnt_rs_server_submit(srv, dict(op="encode", n=65536, k=32768, W=64, seed=1))
        assert ei.value.code == -5
        assert pkg.fnt_rs_server_stats(srv)["rejected"] == 1
    finally:
        pkg.fnt_rs_server_destroy(srv)
    reqs = _trace(64)
    arrivals = [q["t"] / 10 for q in reqs]
    # an arena far smaller than the trace's total: admission waits for memory
    total = sum(q["k"] * q["W"] * 2 + q["n"] * q["W"] * 4 for q in reqs)
    srv = pkg.fnt_rs_server_create(96 << 20, nstreams=4, keep_results=False)
    try:
        assert total > 96 << 20
        lat, wall = pkg.fnt_rs_server_replay(srv, reqs, arrivals)
        assert (lat >= 0).all() and wall > 0
        st = pkg.fnt_rs_server_stats(srv)
        assert st["completed"] >= 64 and st["arena_used"] == 0
    finally:
        pkg.fnt_rs_server_destroy(srv)
    lat, wall = pkg.fnt_rs_baseline_replay(reqs[:16], arrivals[:16])
    assert (lat >= 0).all()


def test_replay_latency_counts_from_scheduled_arrival(pkg):
    # Every request is due at once: the last result must arrive about one wall
    # time after the start, so the largest latency (counted from the due time,
    # queueing and late submission included) is close to the replay's wall time,
    # and no latency can be below the shortest possible queue wait of zero.
    reqs = _trace(32)
    arrivals = [0.0] * len(reqs)
    srv = pkg.fnt_rs_server_create(1 << 30, nstreams=4, keep_results=False)
    try:
        for n, k in {(q["n"], q["k"]) for q in reqs}:
            pkg.fnt_rs_server_preplan(srv, n, k)
        lat, wall = pkg.fnt_rs_server_replay(srv, reqs, arrivals)
    finally:
        pkg.fnt_rs_server_destroy(srv)
    assert (lat >= 0).all()
    assert lat.max() <= wall * 1e3 + 1.0
    assert lat.max() >= 0.8 * wall * 1e3 - 1.0
    blat, bwall = pkg.fnt_rs_baseline_replay(reqs, arrivals)
    assert (blat >= 0).all()
    # one request at a time from a common due time: latencies grow in trace order
    assert np.all(np.diff(blat) >= 0)
    assert blat.max() <= bwall * 1e3 + 1.0
