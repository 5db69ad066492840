"""The direct (quadratic) systematic encoder and decoder (Sec. III, Tables I-II)
on the GPU vs the CPU oracle, bit-exact: the same systematic code as the FNT
route (oracle.encode_sys / oracle.decode_sys), computed as products by
Lagrange-basis matrices."""
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


def _direct_plan(pkg, n, k):
    plan = pkg.Plan(n, k)
    plan.set_schedule(pkg.OP_ENCODE_SYS, pkg.SCHED_DIRECT)
    plan.set_schedule(pkg.OP_DECODE_SYS, pkg.SCHED_DIRECT)
    assert plan.schedule(pkg.OP_ENCODE_SYS) == pkg.SCHED_DIRECT
    return plan


@pytest.mark.parametrize("n,k,W", [(2, 1, 3), (16, 5, 9), (64, 20, 70), (512, 256, 130),
                                   (1024, 1000, 16), (4096, 1024, 8)])
def test_direct_encode_matches_oracle(pkg, n, k, W):
    src = synth.source(n + k, k, W)
    plan = _direct_plan(pkg, n, k)
    enc = pkg.to_host(plan.encode_sys(pkg.to_device(src)))
    assert np.array_equal(enc, oracle.encode_sys(src, n))
    assert plan.status() == 0


@pytest.mark.parametrize("n,k,W", [(16, 5, 9), (64, 20, 70), (512, 256, 130), (4096, 1024, 8)])
def test_direct_decode_matches_oracle(pkg, n, k, W):
    seed = 3 * n + k
    plan = _direct_plan(pkg, n, k)
    src = synth.source(seed, k, W)
    enc = pkg.to_host(plan.encode_sys(pkg.to_device(src)))
    for kind in ("uniform", "burst"):
        er = (synth.erased_uniform if kind == "uniform" else synth.erased_burst)(seed + 1, n, k)
        pos = synth.received_positions(n, er)
        out = pkg.to_host(plan.decode_sys(pkg.to_device(np.ascontiguousarray(enc[pos])), pos))
        assert np.array_equal(out, src), kind
    assert plan.status() == 0
    # arbitrary received words: the interpolant's values at r^0..r^(k-1)
    rng = np.random.default_rng(seed)
    pos = rng.permutation(n)[:k].astype(np.uint32)
    v = rng.integers(0, P, (k, W), dtype=np.uint32)
    got = pkg.to_host(plan.decode_sys(pkg.to_device(v), pos))
    want, flag = oracle.decode_sys(v, pos, n, k)
    assert np.array_equal(got, want)
    assert (plan.status() == pkg.E_RANGE) == flag


def test_direct_equals_fnt_route_punctured_and_patterns(pkg):
    n, k, W, n_out = 1024, 300, 40, 700
    src = synth.source(5, k, W)
    fnt = pkg.Plan(n, k)
    fnt.set_length(n_out)
    plan = _direct_plan(pkg, n, k)
    plan.set_length(n_out)
    e1 = pkg.to_host(plan.encode_sys(pkg.to_device(src)))
    e2 = pkg.to_host(fnt.encode_sys(pkg.to_device(src)))
    assert e1.shape[0] == n_out and np.array_equal(e1, e2)
    rng = np.random.default_rng(6)
    for _ in range(3):  # new patterns rebuild the decode matrix
        pos = rng.permutation(n_out)[:k].astype(np.uint32)
        d1 = pkg.to_host(plan.decode_sys(pkg.to_device(np.ascontiguousarray(e1[pos])), pos))
        assert np.array_equal(d1, src)
    # all source positions lost
    pos = np.arange(k, n_out, dtype=np.uint32)[:k]
    assert np.array_equal(pkg.to_host(plan.decode_sys(
        pkg.to_device(np.ascontiguousarray(e1[pos])), pos)), src)
    assert plan.status() == 0


def test_direct_availability_and_switch_back(pkg):
    plan = pkg.Plan(4096, 2048)  # k above the direct limit
    with pytest.raises(pkg.FntRsError):
        plan.set_schedule(pkg.OP_ENCODE_SYS, pkg.SCHED_DIRECT)
    with pytest.raises(pkg.FntRsError):
        plan.set_schedule(pkg.OP_ENCODE, pkg.SCHED_DIRECT)  # the non-systematic ones too
    with pytest.raises(pkg.FntRsError):
        pkg.Plan(256, 100).set_schedule(pkg.OP_FNT, pkg.SCHED_DIRECT)  # not an op with schedules
    plan = _direct_plan(pkg, 256, 100)
    plan.set_schedule(pkg.OP_ENCODE_SYS, pkg.SCHED_AUTO)
    assert plan.schedule(pkg.OP_ENCODE_SYS) != pkg.SCHED_DIRECT
    src = synth.source(9, 100, 12)
    assert np.array_equal(pkg.to_host(plan.encode_sys(pkg.to_device(src))),
                          oracle.encode_sys(src, 256))


def test_tensor_core_and_integer_products_agree(pkg, monkeypatch):
    """The direct methods run their matrix products on the tensor cores (BF16 limbs,
    exact FP32 accumulation); FNTRS_DIRECT_SIMT=1 selects the integer kernel.  Both
    must give the oracle's words, at the largest k the exactness bound allows."""
    n, k, W = 2048, 1024, 136
    src = synth.source(77, k, W)
    want = oracle.encode_sys(src, n)
    pos = synth.received_positions(n, synth.erased_uniform(78, n, k))
    v = synth.received_uniform(79, k, W)
    want_d, _ = oracle.decode_sys(v, pos, n, k)
    for simt in ("0", "1"):
        monkeypatch.setenv("FNTRS_DIRECT_SIMT", simt)
        plan = _direct_plan(pkg, n, k)
        assert np.array_equal(pkg.to_host(plan.encode_sys(pkg.to_device(src))), want), simt
        got = pkg.to_host(plan.decode_sys(pkg.to_device(v), pos))
        assert np.array_equal(got, want_d), simt
        plan.status()


def _direct_code_plan(pkg, n, k):
    plan = pkg.Plan(n, k)
    plan.set_schedule(pkg.OP_ENCODE, pkg.SCHED_DIRECT)
    plan.set_schedule(pkg.OP_DECODE, pkg.SCHED_DIRECT)
    assert plan.schedule(pkg.OP_DECODE) == pkg.SCHED_DIRECT
    return plan


@pytest.mark.parametrize("n,k,W", [(2, 1, 3), (16, 5, 9), (64, 20, 70), (512, 256, 130),
                                   (2048, 1024, 40), (16384, 256, 8)])
def test_direct_nonsystematic_code_matches_oracle(pkg, n, k, W):
    """Encode e = V s with V[j][i] = r^(ij) and decode s = M v with M the Lagrange-basis
    coefficients of the received points, as tensor-core products (Sec. II.A's matrix view
    of the code, Sec. III's quadratic methods)."""
    seed = 7 * n + k
    src = synth.source(seed, k, W)
    plan = _direct_code_plan(pkg, n, k)
    enc = pkg.to_host(plan.encode(pkg.to_device(src)))
    if n <= 2048:
        assert np.array_equal(enc, oracle.encode(src, n))
    else:
        rows = np.array([0, 1, n // 2, n - 1], np.uint32)
        assert np.array_equal(enc[rows], oracle.encode_rows(src, n, rows))
    pos = synth.received_positions(n, synth.erased_uniform(seed + 1, n, k))
    assert np.array_equal(pkg.to_host(plan.decode(pkg.to_device(np.ascontiguousarray(enc[pos])),
                                                  pos)), src)
    assert plan.status() == 0
    v = synth.received_uniform(seed + 2, k, W)
    got = pkg.to_host(plan.decode(pkg.to_device(v), pos))
    want, flag = oracle.decode(v, pos, n, k)
    assert np.array_equal(got, want)
    assert (plan.status() == pkg.E_RANGE) == flag


def test_direct_code_slots_systematic_punctured_and_tuner(pkg):
    n, k, W = 1024, 300, 72
    src = synth.source(91, k, W)
    plan = _direct_code_plan(pkg, n, k)
    enc = pkg.to_host(plan.encode(pkg.to_device(src)))
    pos = synth.received_positions(n, synth.erased_burst(92, n, k))
    # slot buffer: row z = position z
    assert np.array_equal(pkg.to_host(plan.decode_slots(pkg.to_device(enc), pos)), src)
    # the systematic FNT route interpolates through the decode schedule (u32 coefficients)
    es = pkg.to_host(plan.encode_sys(pkg.to_device(src)))
    assert np.array_equal(es, oracle.encode_sys(src, n))
    # punctured: the direct product writes the first n_out rows
    plan.set_length(700)
    e2 = pkg.to_host(plan.encode(pkg.to_device(src)))
    assert e2.shape[0] == 700 and np.array_equal(e2, enc[:700])
    plan.set_length(n)
    assert plan.status() == 0
    # the tuner times the transform schedules only: the plain code never moves to
    # the tensor-core product unless the caller asks for it
    t = pkg.Plan(512, 128)
    for op in (pkg.OP_ENCODE, pkg.OP_DECODE):
        res = t.autotune(256, op)
        assert res and pkg.SCHED_DIRECT not in [r[0] for r in res]
        assert t.schedule(op) != pkg.SCHED_DIRECT
    src2 = synth.source(93, 128, 256)
    e3 = pkg.to_host(t.encode(pkg.to_device(src2)))
    assert np.array_equal(e3, oracle.encode(src2, 512))
    pos2 = synth.received_positions(512, synth.erased_uniform(94, 512, 128))
    assert np.array_equal(pkg.to_host(t.decode(pkg.to_device(np.ascontiguousarray(e3[pos2])),
                                               pos2)), src2)
