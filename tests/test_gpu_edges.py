"""Degenerate batches on the GPU: no codewords (W = 0) is a no-op for every call
(status OK, nothing launched, outputs untouched); the smallest code (n = 2,
k = 1) and k = n (nothing erased: any n positions) through every entry point."""
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


def test_empty_batches_are_no_ops(pkg):
    n, k = 1024, 300
    plan = pkg.Plan(n, k)
    pos = np.arange(k, dtype=np.uint32)
    src = torch.zeros((k, 0), dtype=torch.int16, device="cuda")
    enc = torch.zeros((n, 0), dtype=torch.int32, device="cuda")
    out = torch.zeros((k, 0), dtype=torch.int16, device="cuda")
    sentinel = torch.full((4,), 7, dtype=torch.int32, device="cuda")
    before = pkg.fnt_rs_launch_count()
    pkg.fnt_rs_encode(plan.handle, src, enc, None)
    pkg.fnt_rs_decode(plan.handle, enc[:k], pos, out, None)  # builds the pattern, then nothing
    pkg.fnt_rs_fnt(plan.handle, enc, enc.clone(), False, None)
    pkg.fnt_rs_encode_sys(plan.handle, src, enc, None)
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    esc = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    pkg.fnt_rs_encode_wire(plan.handle, src, torch.zeros((n, 0), dtype=torch.int16,
                                                          device="cuda"), esc, cnt, None)
    torch.cuda.synchronize()
    launched = pkg.fnt_rs_launch_count() - before
    assert launched <= 1  # at most the pattern build of the decode
    assert int(cnt.item()) == 0 and int(sentinel.sum().item()) == 28
    assert plan.status() == 0


@pytest.mark.parametrize("n,k,W", [(2, 1, 5), (2, 2, 3), (16, 16, 7), (8192, 8192, 16)])
def test_smallest_and_full_rate_codes(pkg, n, k, W):
    src = synth.source(n + k, k, W)
    plan = pkg.Plan(n, k)
    enc = pkg.to_host(plan.encode(pkg.to_device(src)))
    if n <= 16:
        assert np.array_equal(enc, oracle.encode(src, n))
    pos = np.random.default_rng(n).permutation(n)[:k].astype(np.uint32)
    out = pkg.to_host(plan.decode(pkg.to_device(np.ascontiguousarray(enc[pos])), pos))
    assert np.array_equal(out, src)
    es = pkg.to_host(plan.encode_sys(pkg.to_device(src)))
    assert np.array_equal(es[:k], src.astype(np.uint32))
    assert np.array_equal(pkg.to_host(plan.decode_sys(
        pkg.to_device(np.ascontiguousarray(es[pos])), pos)), src)
    sym, esc = plan.encode_wire(pkg.to_device(src))
    assert np.array_equal(pkg.to_host(sym), (enc & 0xFFFF).astype(np.uint16))
    assert plan.status() == 0
