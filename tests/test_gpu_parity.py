"""GPU path vs the CPU oracle, bit-exact (the arithmetic is exact mod p).

Every call goes through the C ABI (libfntrs.so) via the thin binding.  Small
cases are compared element by element in full; large ones on seeded column
samples the oracle can afford, plus properties that hold at any size
(decode(encode(s)) == s on every codeword, IFNT(FNT(x)) == x).
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

P = 65537


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


def _enc(pkg, plan, src):
    return pkg.to_host(plan.encode(pkg.to_device(src)))


def _dec(pkg, plan, recv, pos):
    return pkg.to_host(plan.decode(pkg.to_device(recv), pos))


# ---------------------------------------------------------------- encode
@pytest.mark.parametrize("n,k,W", [
    (2, 1, 5), (2, 2, 3), (4, 3, 7), (8, 8, 9), (16, 5, 33), (32, 16, 130),
    (64, 32, 64), (64, 63, 17), (128, 100, 40), (256, 128, 300), (512, 256, 512),
    (512, 511, 20), (1024, 700, 70), (2048, 1024, 35), (4096, 2048, 19), (4096, 4096, 9),
    (8192, 4096, 13), (8192, 5000, 5), (8192, 1, 3),
])
def test_encode_matches_oracle(pkg, n, k, W):
    src = synth.source(n + k + W, k, W)
    plan = pkg.Plan(n, k)
    got = _enc(pkg, plan, src)
    assert np.array_equal(got, oracle.encode(src, n))


@pytest.mark.parametrize("n,k,W", [(16384, 8192, 24), (32768, 12345, 9), (65536, 32768, 16),
                                   (65536, 65536, 3)])
def test_encode_split_sizes_sampled(pkg, n, k, W):
    src = synth.source(7 * n + k, k, W)
    plan = pkg.Plan(n, k)
    got = _enc(pkg, plan, src)
    rng = np.random.default_rng(n + W)
    rows = np.sort(rng.choice(n, 8, replace=False)).astype(np.uint32)
    assert np.array_equal(got[rows], oracle.encode_rows(src, n, rows))
    cols = [0, W - 1]
    assert np.array_equal(got[:, cols], oracle.encode(src[:, cols], n))


@pytest.mark.parametrize("n,k,W", [(64, 40, 48), (512, 256, 72), (1024, 1000, 40),
                                   (2048, 1024, 24), (4096, 4000, 16), (4096, 4096, 64),
                                   (8192, 4096, 40), (8192, 3000, 24), (8192, 4096, 2048)])
def test_encode_tma_and_fallback_paths(pkg, n, k, W, monkeypatch):
    # aligned widths take the TMA-staged persistent kernel, FNTRS_NO_TMA the generic one
    src = synth.source(5 * n + k + W, k, W)
    cols = slice(None) if W <= 64 else [0, 1, W // 2, W - 1]
    want = oracle.encode(np.ascontiguousarray(src[:, cols]), n)
    got_tma = _enc(pkg, pkg.Plan(n, k), src)
    monkeypatch.setenv("FNTRS_NO_TMA", "1")
    got_gen = _enc(pkg, pkg.Plan(n, k), src)
    assert np.array_equal(got_tma[:, cols], want)
    assert np.array_equal(got_gen, got_tma)


def test_encode_leading_dimensions(pkg):
    n, k, W = 1024, 512, 100
    src = synth.source(9, k, W)
    wide = np.zeros((k, W + 28), dtype=np.uint16)
    wide[:, 5:5 + W] = src
    d_wide = pkg.to_device(wide)
    out_wide = torch.zeros((n, W + 40), dtype=torch.int32, device="cuda")
    plan = pkg.Plan(n, k)
    pkg.fnt_rs_encode(plan.handle, d_wide[:, 5:5 + W], out_wide[:, 3:3 + W])
    got = pkg.to_host(out_wide)
    assert np.array_equal(got[:, 3:3 + W], oracle.encode(src, n))
    assert not got[:, :3].any() and not got[:, 3 + W:].any()


def test_custom_root(pkg):
    n, k, W = 64, 40, 12
    r = oracle.root(n)
    root = pow(r, 5, P)  # another root of order n: a different (still MDS) code
    src = synth.source(31, k, W)
    plan = pkg.Plan(n, k, root=root)
    got = _enc(pkg, plan, src)
    assert np.array_equal(got, oracle.encode(src, n, root_=root))
    pos = synth.received_positions(n, synth.erased_uniform(32, n, k))
    assert np.array_equal(_dec(pkg, plan, got[pos], pos), src)
    v = synth.received_uniform(33, k, W)
    want, _ = oracle.decode(v, pos, n, k, root_=root)
    assert np.array_equal(_dec(pkg, plan, v, pos), want)


# ---------------------------------------------------------------- FNT
@pytest.mark.parametrize("n,W", [(2, 3), (8, 5), (32, 40), (64, 9), (256, 33), (1024, 6),
                                 (4096, 3), (8192, 2)])
def test_fnt_matches_dft_definition(pkg, n, W):
    rng = np.random.default_rng(n)
    x = rng.integers(0, 1 << 32, size=(n, W), dtype=np.uint64).astype(np.uint32)
    plan = pkg.Plan(n, 1)
    fwd = pkg.to_host(plan.fnt(pkg.to_device(x)))
    inv = pkg.to_host(plan.fnt(pkg.to_device(x), inverse=True))
    xm = (x % P).astype(np.uint32)
    assert np.array_equal(fwd, oracle.dft(xm))
    assert np.array_equal(inv, oracle.dft(xm, inverse=True))


@pytest.mark.parametrize("n,W", [(16384, 5), (32768, 3), (65536, 4)])
def test_fnt_split_roundtrip_and_encode_consistency(pkg, n, W):
    rng = np.random.default_rng(n)
    x = rng.integers(0, P, size=(n, W), dtype=np.uint32)
    plan = pkg.Plan(n, n // 2)
    fx = plan.fnt(pkg.to_device(x))
    back = pkg.to_host(plan.fnt(fx, inverse=True))
    assert np.array_equal(back, x)
    # FNT of a zero-padded 16-bit vector is its encoding (Sec. II.B)
    src = synth.source(n + 1, n // 2, W)
    pad = np.zeros((n, W), dtype=np.uint32)
    pad[: n // 2] = src
    f = pkg.to_host(plan.fnt(pkg.to_device(pad)))
    rows = np.sort(rng.choice(n, 6, replace=False)).astype(np.uint32)
    assert np.array_equal(f[rows], oracle.encode_rows(src, n, rows))


# ---------------------------------------------------------------- decode
@pytest.mark.parametrize("n,k,W", [
    (2, 1, 3), (4, 2, 5), (8, 3, 9), (8, 5, 9), (16, 8, 17), (16, 15, 4), (32, 16, 40),
    (32, 31, 8), (64, 16, 33), (64, 32, 64), (64, 48, 20), (128, 64, 50), (256, 128, 130),
    (256, 200, 20), (512, 256, 64), (512, 448, 16), (1024, 512, 40), (1024, 1024, 4),
    (2048, 1024, 17), (2048, 1536, 8), (4096, 2048, 9), (4096, 3000, 4), (8192, 4096, 9),
    (8192, 6144, 4),
])
def test_decode_random_received_matches_oracle(pkg, n, k, W):
    # any k received values define a unique interpolant (not only codewords)
    seed = 3 * n + k
    rng = np.random.default_rng(seed)
    pos = rng.permutation(n)[:k].astype(np.uint32)  # caller's order, not sorted
    v = synth.received_uniform(seed, k, W)
    plan = pkg.Plan(n, k)
    got = _dec(pkg, plan, v, pos)
    want, flag = oracle.decode(v, pos, n, k)
    assert np.array_equal(got, want)
    st = plan.status()
    assert st == (pkg.E_RANGE if flag else 0)


@pytest.mark.parametrize("n,k,W", [(8192, 4096, 643), (4096, 2048, 1285), (8192, 3000, 645),
                                   (512, 256, 9927)])
def test_decode_full_and_half_width_tiles(pkg, n, k, W):
    # W large enough for a full round of full-width tiles with a short last
    # round, which the staged decode cuts into half-width tiles (and a ragged
    # last tile): every codeword must come back, and random received words
    # must match the oracle in columns of every kind of tile
    src = synth.source(7 * n + W, k, W)
    plan = pkg.Plan(n, k)
    enc = pkg.to_host(plan.encode(pkg.to_device(src)))
    pos = synth.received_positions(n, synth.erased_uniform(n + W, n, k))
    assert np.array_equal(_dec(pkg, plan, np.ascontiguousarray(enc[pos]), pos), src)
    assert plan.status() == 0
    v = synth.received_uniform(W + k, k, W)
    got = _dec(pkg, plan, v, pos)
    cols = sorted({0, 1, W // 2, W - 9, W - 6, W - 5, W - 4, W - 3, W - 1})
    want, flag = oracle.decode(np.ascontiguousarray(v[:, cols]), pos, n, k)
    assert np.array_equal(got[:, cols], want)


@pytest.mark.parametrize("n,k,W,col,extra", [(8192, 4096, 96, 1, 3), (8192, 4096, 64, 4, 4),
                                               (4096, 2048, 72, 2, 6), (8192, 3000, 40, 3, 5),
                                               (1024, 512, 100, 0, 1)])
def test_decode_output_leading_dimensions(pkg, n, k, W, col, extra):
    # the staged decode writes a row's tile columns with one wide store when
    # the row segment is aligned: an output inside a wider matrix, at an odd
    # column or with an odd row length, takes the narrow stores instead
    src = synth.source(13 * n + col, k, W)
    plan = pkg.Plan(n, k)
    enc = pkg.to_host(plan.encode(pkg.to_device(src)))
    pos = synth.received_positions(n, synth.erased_uniform(n + col, n, k))
    d_recv = pkg.to_device(np.ascontiguousarray(enc[pos]))
    wide = torch.zeros((k, W + col + extra), dtype=torch.int16, device="cuda")
    pkg.fnt_rs_decode(plan.handle, d_recv, pos, wide[:, col:col + W])
    got = pkg.to_host(wide)
    assert np.array_equal(got[:, col:col + W], src)
    assert not got[:, :col].any() and not got[:, col + W:].any()
    assert plan.status() == 0
    v = synth.received_uniform(W + col, k, W)
    wide.zero_()
    pkg.fnt_rs_decode(plan.handle, pkg.to_device(v), pos, wide[:, col:col + W])
    got = pkg.to_host(wide)[:, col:col + W]
    cols = [0, 1, W // 2, W - 2, W - 1]
    want, _ = oracle.decode(np.ascontiguousarray(v[:, cols]), pos, n, k)
    assert np.array_equal(got[:, cols], want)


@pytest.mark.parametrize("n,k,W", [(16384, 8192, 8), (16384, 12000, 5), (65536, 32768, 3),
                                   (32768, 30000, 3), (32768, 16384, 4), (32768, 10000, 3)])
def test_decode_split_sizes_sampled(pkg, n, k, W):
    seed = n + k
    rng = np.random.default_rng(seed)
    pos = rng.permutation(n)[:k].astype(np.uint32)
    v = synth.received_uniform(seed, k, W)
    plan = pkg.Plan(n, k)
    got = _dec(pkg, plan, v, pos)
    cols = [0, W - 1]
    want, _ = oracle.decode(v[:, cols], pos, n, k)
    assert np.array_equal(got[:, cols], want)


@pytest.mark.parametrize("n,k,W", [(16384, 8192, 64), (65536, 32768, 16), (32768, 28672, 8),
                                   (32768, 16384, 6), (16384, 12000, 16), (8192, 7168, 32),
                                   (256, 224, 200)])
def test_roundtrip_every_codeword(pkg, n, k, W):
    src = synth.source(n * 3 + 1, k, W)
    plan = pkg.Plan(n, k)
    enc = plan.encode(pkg.to_device(src))
    enc_h = pkg.to_host(enc)
    pos = synth.received_positions(n, synth.erased_uniform(n + 5, n, k))
    out = _dec(pkg, plan, enc_h[pos], pos)
    assert np.array_equal(out, src)
    assert plan.status() == 0


@pytest.mark.parametrize("n,k,W", [(64, 32, 36), (256, 100, 68), (1024, 512, 40),
                                   (2048, 1024, 20), (4096, 2048, 24), (8192, 4096, 12),
                                   (8192, 4096, 2048), (8192, 6000, 8), (16384, 8192, 8),
                                   (16384, 12000, 4), (32768, 16000, 4)])
@pytest.mark.parametrize("route", ["log", "tree"])
def test_decode_paths_and_plan_routes(pkg, n, k, W, route, monkeypatch):
    # plan tables by the log-domain correlation (default) or the product tree;
    # aligned widths take the TMA-staged persistent decode, FNTRS_NO_TMA the generic one
    if route == "tree":
        monkeypatch.setenv("FNTRS_PLAN", "tree")
    seed = 11 * n + k + W
    src = synth.source(seed, k, W)
    pos = synth.received_positions(n, synth.erased_uniform(seed + 1, n, k))
    plan = pkg.Plan(n, k)
    enc_h = _enc(pkg, plan, src)
    assert np.array_equal(_dec(pkg, plan, enc_h[pos], pos), src)
    v = synth.received_uniform(seed + 2, k, W)
    got = _dec(pkg, plan, v, pos)
    cols = slice(None) if W <= 64 else [0, 1, W - 2, W - 1]
    want, _ = oracle.decode(np.ascontiguousarray(v[:, cols]), pos, n, k)
    assert np.array_equal(got[:, cols], want)
    monkeypatch.setenv("FNTRS_NO_TMA", "1")
    plan2 = pkg.Plan(n, k)
    assert np.array_equal(_dec(pkg, plan2, v, pos), got)


def test_extra_positions_use_first_k(pkg):
    n, k, W = 256, 100, 30
    src = synth.source(44, k, W)
    plan = pkg.Plan(n, k)
    enc_h = _enc(pkg, plan, src)
    rng = np.random.default_rng(44)
    pos = rng.permutation(n)[: k + 37].astype(np.uint32)
    assert np.array_equal(_dec(pkg, plan, enc_h[pos], pos), src)


def test_pattern_cache_cycles(pkg):
    n, k, W = 512, 256, 16
    src = synth.source(55, k, W)
    plan = pkg.Plan(n, k)
    enc_h = _enc(pkg, plan, src)
    pats = [synth.received_positions(n, synth.erased_uniform(60 + i, n, k)) for i in range(6)]
    for rnd in range(2):
        for pos in pats:
            assert np.array_equal(_dec(pkg, plan, enc_h[pos], pos), src)
    assert plan.info()["patterns"] == 4


def test_range_flag_and_zero(pkg):
    n, k, W = 16, 8, 2
    coeffs = np.array([[65536, 1], [5, 2], [6, 3], [7, 4], [8, 5], [9, 6], [10, 7], [11, 65536]],
                      dtype=np.uint32)
    full = np.zeros((n, W), dtype=np.uint32)
    full[:k] = coeffs
    e = oracle.dft(full)
    pos = np.arange(3, 3 + k, dtype=np.uint32)
    plan = pkg.Plan(n, k)
    got = _dec(pkg, plan, e[pos], pos)
    want, flag = oracle.decode(e[pos], pos, n, k)
    assert flag and np.array_equal(got, want)
    assert got[0, 0] == 0 and got[7, 1] == 0
    assert plan.status() == pkg.E_RANGE
    assert plan.status() == 0  # cleared by the read
    bad = e[pos].copy()
    bad[2, 0] = 70000
    _dec(pkg, plan, bad, pos)
    assert plan.status() == pkg.E_RANGE


def test_position_errors(pkg):
    n, k = 64, 8
    plan = pkg.Plan(n, k)
    v = pkg.to_device(np.zeros((k, 4), dtype=np.uint32))
    for pos in ([0, 1, 2, 3, 4, 5, 6, 6], [0, 1, 2, 3, 4, 5, 6, 64], [0, 1, 2]):
        with pytest.raises(pkg.FntRsError) as ei:
            plan.decode(v, np.array(pos, dtype=np.uint32))
        assert ei.value.code == -4


def test_lossless_is_inverse_fnt(pkg):
    n, k, W = 1024, 600, 20
    src = synth.source(77, k, W)
    plan = pkg.Plan(n, k)
    enc_h = _enc(pkg, plan, src)
    allpos = np.arange(n, dtype=np.uint32)
    assert np.array_equal(_dec(pkg, plan, enc_h, allpos), src)
    back = pkg.to_host(plan.fnt(pkg.to_device(enc_h), inverse=True))
    assert np.array_equal(back[:k], src.astype(np.uint32)) and not back[k:].any()


@pytest.mark.parametrize("n,k,W", [(8, 5, 3), (512, 256, 40), (8192, 4096, 24), (16384, 9000, 8),
                                   (65536, 32768, 4)])
def test_lossless_fast_path(pkg, n, k, W):
    # Sec. II.B: nothing lost -> first k outputs of the inverse FNT
    src = synth.source(n + k + 3, k, W)
    plan = pkg.Plan(n, k)
    enc = plan.encode(pkg.to_device(src))
    assert np.array_equal(pkg.to_host(plan.decode_full(enc)), src)
    # arbitrary words: the first k coefficients of the degree < n interpolant
    v = synth.received_uniform(n + 7, n, 2)
    got = pkg.to_host(plan.decode_full(pkg.to_device(v)))
    want = oracle.dft(v, inverse=True)[:k] if n <= 8192 else None
    if want is not None:
        flag = (want == 65536).any()
        assert np.array_equal(got, np.where(want == 65536, 0, want).astype(np.uint16))
        assert plan.status() == (pkg.E_RANGE if flag else 0)


def test_host_buffer_entry_points(pkg):
    n, k, W = 2048, 1024, 48
    src = synth.source(88, k, W)
    plan = pkg.Plan(n, k)
    h_src = torch.from_numpy(src.view(np.int16)).pin_memory()
    h_enc = torch.empty((n, W), dtype=torch.int32).pin_memory()
    ws = plan.workspace(W, pkg.OP_ENCODE_HOST)
    pkg.fnt_rs_encode_host(plan.handle, h_src, h_enc, ws)
    enc_h = h_enc.numpy().view(np.uint32)
    assert np.array_equal(enc_h, oracle.encode(src, n))
    pos = synth.received_positions(n, synth.erased_uniform(89, n, k))
    h_recv = torch.from_numpy(np.ascontiguousarray(enc_h[pos]).view(np.int32)).pin_memory()
    h_out = torch.empty((k, W), dtype=torch.int16).pin_memory()
    ws2 = plan.workspace(W, pkg.OP_DECODE_HOST)
    pkg.fnt_rs_decode_host(plan.handle, h_recv, pos, h_out, ws2)
    assert np.array_equal(h_out.numpy().view(np.uint16), src)


# ---------------------------------------------------------------- workloads
def test_workload_k256_n512_full_oracle(pkg):
    cfg = synth.CONFIGS["k256_n512_w512"]
    src = cfg.source()
    plan = pkg.Plan(cfg.n, cfg.k)
    enc_h = _enc(pkg, plan, src)
    assert np.array_equal(enc_h, oracle.encode(src, cfg.n))
    pos = cfg.positions()
    got = _dec(pkg, plan, enc_h[pos], pos)
    want, flag = oracle.decode(enc_h[pos], pos, cfg.n, cfg.k)
    assert not flag and np.array_equal(got, want) and np.array_equal(got, src)


@pytest.mark.parametrize("name", ["k4096_n8192_w2048", "k32768_n65536_w1024_burst",
                                  "k32768_n65536_w1024_uniform"])
def test_workload_full_size(pkg, name):
    cfg = synth.CONFIGS[name]
    src = cfg.source()
    plan = pkg.Plan(cfg.n, cfg.k)
    d_enc = plan.encode(pkg.to_device(src))
    enc_h = pkg.to_host(d_enc)
    rng = np.random.default_rng(cfg.seed)
    # 4 seeded rows by Horner (O(k) each) on every (W/64)-th codeword, two full
    # codewords by the oracle; the round trip below covers every codeword
    cols = np.sort(rng.choice(cfg.W, 2, replace=False))
    rows = np.sort(rng.choice(cfg.n, 4, replace=False)).astype(np.uint32)
    sub = np.ascontiguousarray(src[:, :: max(1, cfg.W // 64)])
    assert np.array_equal(enc_h[rows][:, :: max(1, cfg.W // 64)], oracle.encode_rows(sub, cfg.n, rows))
    assert np.array_equal(enc_h[:, cols], oracle.encode(np.ascontiguousarray(src[:, cols]), cfg.n))
    pos = cfg.positions()
    out = _dec(pkg, plan, np.ascontiguousarray(enc_h[pos]), pos)
    assert np.array_equal(out, src)  # every codeword
    assert plan.status() == 0
