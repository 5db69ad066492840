"""Tile scheduling of the TMA-staged encode and decode kernels.

Both kernels are launched with one CTA per tile of codewords; a running CTA
cancels the launch of a CTA that has not started and processes its tile
(cluster launch control).  Which CTA transforms a tile must not change any
result: these tests run many tiles per SM, and the encode concurrently with a
decode of the same plan on another stream, and compare bit-exactly with the
generic (non-TMA) kernels and with the oracle on sampled columns.
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


@pytest.mark.parametrize("n,k,W", [(8192, 4096, 8192), (1024, 512, 32768), (256, 128, 65536)])
def test_many_tiles_per_sm(pkg, n, k, W, monkeypatch):
    seed = 3 * n + W
    src = synth.source(seed, k, W)
    pos = synth.received_positions(n, synth.erased_uniform(seed + 1, n, k))
    plan = pkg.Plan(n, k)
    enc = pkg.to_host(plan.encode(pkg.to_device(src)))
    assert plan.status() == 0
    assert np.array_equal(pkg.to_host(plan.decode(pkg.to_device(enc[pos]), pos)), src)
    assert plan.status() == 0
    # arbitrary received words (their decodings may hit 65536: range flag)
    v = synth.received_uniform(seed + 2, k, W)
    dec = pkg.to_host(plan.decode(pkg.to_device(v), pos))
    rng = np.random.default_rng(seed)
    cols = np.sort(rng.choice(W, 3, replace=False))
    assert np.array_equal(enc[:, cols], oracle.encode(np.ascontiguousarray(src[:, cols]), n))
    want, _ = oracle.decode(np.ascontiguousarray(v[:, cols]), pos, n, k)
    assert np.array_equal(dec[:, cols], want)
    # every column against the generic kernels
    monkeypatch.setenv("FNTRS_NO_TMA", "1")
    gen = pkg.Plan(n, k)
    assert np.array_equal(pkg.to_host(gen.encode(pkg.to_device(src))), enc)
    assert np.array_equal(pkg.to_host(gen.decode(pkg.to_device(v), pos)), dec)


@pytest.mark.parametrize("decode_on_main", [True, False])
def test_encode_concurrent_with_decode(pkg, decode_on_main):
    # the bench's step shape: plan + decode of one batch on one stream, encode
    # of another batch on a second stream, same plan
    n, k, W = 8192, 4096, 4096
    dev = torch.device("cuda")
    plan = pkg.Plan(n, k)
    src_a = synth.source(71, k, W)
    src_b = synth.source(72, k, W)
    pats = [synth.received_positions(n, synth.erased_uniform(73 + i, n, k)) for i in range(3)]
    enc_b = pkg.to_host(plan.encode(pkg.to_device(src_b)))
    recvs = [pkg.to_device(np.ascontiguousarray(enc_b[p])) for p in pats]
    d_src = pkg.to_device(src_a)
    d_enc = torch.empty((n, W), dtype=torch.int32, device=dev)
    d_out = torch.empty((k, W), dtype=torch.int16, device=dev)
    ws_e = plan.workspace(W, pkg.OP_ENCODE)
    ws_d = plan.workspace(W, pkg.OP_DECODE)
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream(priority=-1)
    d_st, e_st = (main, side) if decode_on_main else (side, main)
    want_enc = oracle.encode(np.ascontiguousarray(src_a[:, :2]), n)
    serial_enc = pkg.to_host(plan.encode(d_src))
    assert np.array_equal(serial_enc[:, :2], want_enc)
    for rep in range(6):
        d_enc.zero_()
        d_out.zero_()
        fork = torch.cuda.Event()
        fork.record(main)
        side.wait_event(fork)
        pkg.fnt_rs_decode(plan.handle, recvs[rep % 3], pats[rep % 3], d_out, ws_d, d_st)
        pkg.fnt_rs_encode(plan.handle, d_src, d_enc, ws_e, e_st)
        join = torch.cuda.Event()
        join.record(side)
        main.wait_event(join)
        torch.cuda.synchronize()
        assert np.array_equal(pkg.to_host(d_out), src_b), rep
        assert np.array_equal(pkg.to_host(d_enc), serial_enc), rep
    assert plan.status() == 0


# ------------------------------------------------------------------ schedules
@pytest.mark.parametrize("n,k,W", [(1024, 512, 256), (4096, 2000, 37), (8192, 4096, 64), (8192, 4096, 33), (8192, 6000, 32),
                                   (16384, 8192, 24), (16384, 12000, 8), (32768, 16384, 8)])
def test_every_schedule_gives_the_same_words(pkg, n, k, W):
    seed = 17 * n + k
    src = synth.source(seed, k, W)
    pos = synth.received_positions(n, synth.erased_uniform(seed + 1, n, k))
    v = synth.received_uniform(seed + 2, k, W)
    plan = pkg.Plan(n, k)
    encs, decs = {}, {}
    for s in (pkg.SCHED_TMA, pkg.SCHED_CPA, pkg.SCHED_TILE, pkg.SCHED_SPLIT):
        try:
            plan.set_schedule(pkg.OP_ENCODE, s)
        except pkg.FntRsError:
            pass
        else:
            assert plan.schedule(pkg.OP_ENCODE) == s
            encs[s] = pkg.to_host(plan.encode(pkg.to_device(src)))
        try:
            plan.set_schedule(pkg.OP_DECODE, s)
        except pkg.FntRsError:
            pass
        else:
            decs[s] = pkg.to_host(plan.decode(pkg.to_device(v), pos))
    plan.set_schedule(pkg.OP_ENCODE, pkg.SCHED_AUTO)
    plan.set_schedule(pkg.OP_DECODE, pkg.SCHED_AUTO)
    assert len(encs) >= 1 and len(decs) >= 1
    if n > 8192:  # one-CTA tile and split both run (and the staged tile for k <= n/2)
        assert len(encs) == 2 and len(decs) == (3 if (n in (16384, 32768) and 2 * k <= n) else 2)
    first_e, first_d = next(iter(encs.values())), next(iter(decs.values()))
    for e in encs.values():
        assert np.array_equal(e, first_e)
    for d in decs.values():
        assert np.array_equal(d, first_d)
    cols = [0, W - 1]
    assert np.array_equal(first_e[:, cols], oracle.encode(np.ascontiguousarray(src[:, cols]), n))
    want, _ = oracle.decode(np.ascontiguousarray(v[:, cols]), pos, n, k)
    assert np.array_equal(first_d[:, cols], want)


def test_autotune_keeps_the_fastest_schedule(pkg):
    for n, k, W in ((8192, 4096, 512), (16384, 8192, 256), (32768, 16384, 64)):
        plan = pkg.Plan(n, k)
        for op in (pkg.OP_ENCODE, pkg.OP_DECODE):
            res = plan.autotune(W, op)
            assert len(res) >= 1 and all(us > 0 for _, us in res)
            best = min(res, key=lambda r: r[1])[0]
            assert plan.schedule(op) == best
        # the tuned plan still round-trips
        src = synth.source(n, k, W)
        pos = synth.received_positions(n, synth.erased_uniform(n + 3, n, k))
        enc = pkg.to_host(plan.encode(pkg.to_device(src)))
        assert np.array_equal(pkg.to_host(plan.decode(pkg.to_device(enc[pos]), pos)), src)
        assert plan.status() == 0


@pytest.mark.parametrize("k,W", [(4097, 40), (6144, 16), (7000, 9), (8191, 24), (8192, 8)])
def test_high_rate_n8192_encode_folds_on_tma(pkg, k, W):
    """n = 8192, k > 4096: the TMA encode folds rows i and i + 4096 into its two
    output classes; it must give the oracle's words and the generic tile's."""
    n = 8192
    src = synth.source(k + W, k, W)
    plan = pkg.Plan(n, k)
    assert plan.schedule(pkg.OP_ENCODE) == pkg.SCHED_TMA  # the default for these codes now
    enc = pkg.to_host(plan.encode(pkg.to_device(src)))
    cols = sorted({0, W // 2, W - 1})
    rows = np.sort(np.random.default_rng(k).choice(n, 64, replace=False)).astype(np.uint32)
    want = oracle.encode_rows(np.ascontiguousarray(src[:, cols]), n, rows)
    assert np.array_equal(enc[rows][:, cols], want)
    plan.set_schedule(pkg.OP_ENCODE, pkg.SCHED_TILE)
    assert np.array_equal(pkg.to_host(plan.encode(pkg.to_device(src))), enc)
    plan.set_schedule(pkg.OP_ENCODE, pkg.SCHED_AUTO)
    # the 16-bit wire output keeps the generic tile for these codes
    sym, _ = plan.encode_wire(pkg.to_device(src))
    assert np.array_equal(pkg.to_host(sym), (enc & 0xFFFF).astype(np.uint16))
    pos = synth.received_positions(n, synth.erased_uniform(k, n, k))
    out = pkg.to_host(plan.decode(pkg.to_device(np.ascontiguousarray(enc[pos])), pos))
    assert np.array_equal(out, src)
    assert plan.status() == 0
