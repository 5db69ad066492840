"""The paper's decode route on the GPU (schedule FNT_RS_SCHED_PAPER) vs the CPU oracle.

Step 3 by the chirp, step 5 as a middle product and step 6 as a product, all at
length 2n (Sec. II.B and III).  The result is the same interpolant as the
default decode, so the oracle is the plain Lagrange decode; bit-exact.
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


def _paper_plan(pkg, n, k):
    plan = pkg.Plan(n, k)
    plan.set_schedule(pkg.OP_DECODE, pkg.SCHED_PAPER)
    assert plan.schedule(pkg.OP_DECODE) == pkg.SCHED_PAPER
    return plan


@pytest.mark.parametrize("n,k,W", [(2, 1, 5), (16, 5, 9), (64, 20, 17), (512, 256, 40),
                                   (4096, 2000, 24), (8192, 4096, 40), (32768, 16384, 4)])
def test_paper_route_matches_oracle(pkg, n, k, W):
    seed = 13 * n + k
    plan = _paper_plan(pkg, n, k)
    pos = synth.received_positions(n, synth.erased_uniform(seed, n, k))
    v = synth.received_uniform(seed + 1, k, W)
    got = pkg.to_host(plan.decode(pkg.to_device(v), pos))
    c = slice(None) if n <= 8192 else [0, W - 1]
    want, flag = oracle.decode(np.ascontiguousarray(v[:, c]), pos, n, k)
    assert np.array_equal(got[:, c], want)
    st = plan.status()  # E_RANGE iff some coefficient was 65536 (all columns at n <= 8192)
    if c == slice(None):
        assert (st == pkg.E_RANGE) == flag
    # round trip on codewords
    src = synth.source(seed + 2, k, W)
    enc = pkg.to_host(plan.encode(pkg.to_device(src)))
    out = pkg.to_host(plan.decode(pkg.to_device(np.ascontiguousarray(enc[pos])), pos))
    assert np.array_equal(out, src)
    assert plan.status() == 0


def test_paper_route_equals_default_route_and_patterns_cycle(pkg):
    n, k, W = 1024, 400, 33
    plan = _paper_plan(pkg, n, k)
    ref = pkg.Plan(n, k)
    rng = np.random.default_rng(8)
    pats = [rng.permutation(n)[:k].astype(np.uint32) for _ in range(6)]  # > 4 cached slots
    for it in range(2):
        for pos in pats:
            v = rng.integers(0, P, (k, W), dtype=np.uint32)
            a = pkg.to_host(plan.decode(pkg.to_device(v), pos))
            b = pkg.to_host(ref.decode(pkg.to_device(v), pos))
            assert np.array_equal(a, b)
    plan.status()


def test_paper_route_slots_and_systematic(pkg):
    n, k, W = 2048, 1000, 16
    plan = _paper_plan(pkg, n, k)
    src = synth.source(41, k, W)
    enc = pkg.to_host(plan.encode(pkg.to_device(src)))
    pos = synth.received_positions(n, synth.erased_burst(42, n, k))
    out = pkg.to_host(plan.decode_slots(pkg.to_device(enc), pos))
    assert np.array_equal(out, src)
    # the systematic code interpolates through the decode schedule
    es = pkg.to_host(plan.encode_sys(pkg.to_device(src)))
    assert np.array_equal(es, oracle.encode_sys(src, n))
    assert np.array_equal(pkg.to_host(plan.decode_sys(
        pkg.to_device(np.ascontiguousarray(es[pos])), pos)), src)
    assert plan.status() == 0


def test_paper_route_availability(pkg):
    for n, k in [(1024, 600), (65536, 1000)]:  # k > n/2; no root of order 2n
        plan = pkg.Plan(n, k)
        with pytest.raises(pkg.FntRsError):
            plan.set_schedule(pkg.OP_DECODE, pkg.SCHED_PAPER)
    plan = _paper_plan(pkg, 256, 100)
    plan.set_schedule(pkg.OP_DECODE, pkg.SCHED_AUTO)  # back to the default route
    assert plan.schedule(pkg.OP_DECODE) != pkg.SCHED_PAPER
