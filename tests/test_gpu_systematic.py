"""Systematic code and punctured lengths on the GPU vs the CPU oracle, bit-exact.

Systematic encode: interpolate the source at r^0..r^(k-1), transform the
intermediate symbols; the first k rows of the codeword are the source.
Systematic decode: interpolate the first k received points, transform, keep
rows 0..k-1 (copied straight through when the first k positions are 0..k-1).
Puncturing keeps the first n_out positions.
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


def _cols(W):
    return slice(None) if W <= 24 else [0, 1, W // 2, W - 1]


@pytest.mark.parametrize("n,k,W", [(64, 20, 17), (512, 256, 40), (4096, 3000, 24),
                                   (8192, 4096, 64), (16384, 12000, 6), (32768, 16384, 4),
                                   (65536, 32768, 3)])
def test_encode_sys_matches_oracle(pkg, n, k, W):
    src = synth.source(3 * n + k, k, W)
    plan = pkg.Plan(n, k)
    enc = pkg.to_host(plan.encode_sys(pkg.to_device(src)))
    assert np.array_equal(enc[:k], src.astype(np.uint32))  # the systematic rows
    c = _cols(W)
    want = oracle.encode_sys(np.ascontiguousarray(src[:, c]), n)
    assert np.array_equal(enc[:, c], want)
    assert plan.status() == 0


@pytest.mark.parametrize("n,k,W", [(64, 20, 17), (512, 256, 40), (8192, 4096, 64),
                                   (8192, 6000, 16), (16384, 12000, 6), (65536, 32768, 3)])
def test_decode_sys_round_trip_and_oracle(pkg, n, k, W):
    seed = 5 * n + k
    src = synth.source(seed, k, W)
    plan = pkg.Plan(n, k)
    enc = pkg.to_host(plan.encode_sys(pkg.to_device(src)))
    pos = synth.received_positions(n, synth.erased_uniform(seed + 1, n, k))
    out = pkg.to_host(plan.decode_sys(pkg.to_device(np.ascontiguousarray(enc[pos])), pos))
    assert np.array_equal(out, src)
    assert plan.status() == 0
    # arbitrary received words: the interpolant's values at r^0..r^(k-1)
    v = synth.received_uniform(seed + 2, k, W)
    got = pkg.to_host(plan.decode_sys(pkg.to_device(v), pos))
    c = _cols(W)
    want, _ = oracle.decode_sys(np.ascontiguousarray(v[:, c]), pos, n, k)
    assert np.array_equal(got[:, c], want)


def test_decode_sys_direct_and_reordered(pkg):
    n, k, W = 1024, 300, 33
    src = synth.source(7, k, W)
    plan = pkg.Plan(n, k)
    enc = pkg.to_host(plan.encode_sys(pkg.to_device(src)))
    direct = np.arange(k, dtype=np.uint32)  # every source position received first, in order
    out = pkg.to_host(plan.decode_sys(pkg.to_device(np.ascontiguousarray(enc[:k])), direct))
    assert np.array_equal(out, src)
    # the same positions in another order go through interpolation
    perm = np.random.default_rng(1).permutation(k).astype(np.uint32)
    out2 = pkg.to_host(plan.decode_sys(pkg.to_device(np.ascontiguousarray(enc[perm])), perm))
    assert np.array_equal(out2, src)
    # some source positions lost, parity positions used instead
    pos = np.concatenate([np.arange(1, k, dtype=np.uint32), np.array([n - 1], np.uint32)])
    out3 = pkg.to_host(plan.decode_sys(pkg.to_device(np.ascontiguousarray(enc[pos])), pos))
    assert np.array_equal(out3, src)
    assert plan.status() == 0


def test_decode_sys_every_schedule(pkg):
    n, k, W = 16384, 8192, 8
    src = synth.source(11, k, W)
    pos = synth.received_positions(n, synth.erased_uniform(12, n, k))
    plan = pkg.Plan(n, k)
    encs, decs = [], []
    for s in (pkg.SCHED_TILE, pkg.SCHED_SPLIT):
        plan.set_schedule(pkg.OP_DECODE, s)  # the interpolation step of both directions
        e = pkg.to_host(plan.encode_sys(pkg.to_device(src)))
        encs.append(e)
        decs.append(pkg.to_host(plan.decode_sys(pkg.to_device(np.ascontiguousarray(e[pos])),
                                                pos)))
    assert np.array_equal(encs[0], encs[1])
    assert np.array_equal(decs[0], src) and np.array_equal(decs[1], src)


@pytest.mark.parametrize("n,k,n_out,W", [(64, 20, 45, 9), (1024, 512, 700, 40),
                                         (8192, 4096, 6000, 32), (65536, 32768, 40000, 2)])
def test_punctured_code(pkg, n, k, n_out, W):
    seed = n_out + k
    src = synth.source(seed, k, W)
    plan = pkg.Plan(n, k)
    plan.set_length(n_out)
    enc = pkg.to_host(plan.encode(pkg.to_device(src)))
    assert enc.shape[0] == n_out
    c = _cols(W)
    rows = np.sort(np.random.default_rng(seed).choice(n_out, 6, replace=False)).astype(np.uint32)
    assert np.array_equal(enc[rows][:, c], oracle.encode_rows(np.ascontiguousarray(src[:, c]),
                                                              n, rows))
    # any k of the n_out kept positions decode (MDS)
    pos = np.random.default_rng(seed + 1).permutation(n_out)[:k].astype(np.uint32)
    assert np.array_equal(pkg.to_host(plan.decode(pkg.to_device(np.ascontiguousarray(enc[pos])),
                                                  pos)), src)
    # systematic and punctured together
    es = pkg.to_host(plan.encode_sys(pkg.to_device(src)))
    assert es.shape[0] == n_out
    assert np.array_equal(es[:, c], oracle.encode_sys(np.ascontiguousarray(src[:, c]), n, n_out))
    assert np.array_equal(pkg.to_host(plan.decode_sys(
        pkg.to_device(np.ascontiguousarray(es[pos])), pos)), src)
    assert plan.status() == 0
    # positions at or beyond n_out do not exist
    bad = pos.copy()
    bad[0] = n_out
    with pytest.raises(pkg.FntRsError):
        plan.decode(pkg.to_device(np.ascontiguousarray(enc[pos])), bad)
    # the lossless path needs all n positions
    with pytest.raises(pkg.FntRsError):
        plan.decode_full(torch.zeros((n, W), dtype=torch.int32, device="cuda"))
    plan.set_length(n)  # back to the full code
    assert np.array_equal(pkg.to_host(plan.encode(pkg.to_device(src)))[:n_out], enc)
