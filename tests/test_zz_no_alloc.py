"""The allocation-free encode entry point (collected last on purpose).

fnt_rs_encode_noalloc serves callers that cannot allocate device memory once
running -- all memory reserved at start-up, or no cudaMalloc allowed on the
hot path -- by taking the long-code encoder's scratch from a fixed device
array inside the library.  Its output must equal the regular entry point's
(bit-exact, as every result of this library), call after call, since calls
reuse the same scratch.
"""
import numpy as np
import pytest
import torch

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
    return pkg


@pytest.mark.parametrize("n,k,W", [(16384, 8192, 40), (65536, 32768, 64), (32768, 30000, 24)])
def test_noalloc_matches_regular_encode_twice(pkg, n, k, W):
    plan = pkg.Plan(n, k)
    for call in range(2):  # two calls in a row share the scratch array
        src = pkg.to_device(synth.source(1000 * call + n + W, k, W))
        want = plan.encode(src)  # regular entry point, caller workspace
        got = torch.full((n, W), -1, dtype=torch.int32, device="cuda")
        pkg.fnt_rs_encode_noalloc(plan.handle, src, got)
        torch.cuda.synchronize()
        assert torch.equal(got, want)


def test_noalloc_short_code_and_size_limit(pkg):
    plan = pkg.Plan(4096, 2048)
    src = pkg.to_device(synth.source(5, 2048, 16))
    got = torch.empty((4096, 16), dtype=torch.int32, device="cuda")
    pkg.fnt_rs_encode_noalloc(plan.handle, src, got)
    assert torch.equal(got, plan.encode(src))
    big = pkg.Plan(65536, 32768)
    W = pkg.NOALLOC_SCRATCH_BYTES // (65536 * 4) + 1  # one column too many
    src = torch.zeros((32768, W), dtype=torch.int16, device="cuda")
    out = torch.empty((65536, W), dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.FntRsError) as ei:
        pkg.fnt_rs_encode_noalloc(big.handle, src, out)
    assert ei.value.code == -9


def test_noalloc_punctured_long_code_refused_beyond_scratch(pkg):
    # A punctured code is encoded at full length into a buffer of n * W words,
    # with the long code's two-pass scratch behind it: about twice n * W * 4
    # bytes.  Here n * W * 4 is just above 8 MiB, so the whole workspace is
    # above the 16 MiB array and the call must be refused before any launch.
    n, k, n_out = 16384, 8192, 12000
    plan = pkg.Plan(n, k)
    plan.set_length(n_out)
    W = (8 << 20) // (n * 4) + 8
    need = pkg.fnt_rs_workspace_bytes(plan.handle, W, pkg.OP_ENCODE)
    assert n * W * 4 <= pkg.NOALLOC_SCRATCH_BYTES < need
    src = pkg.to_device(synth.source(11, k, W))
    out = torch.full((n_out, W), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    before = pkg.fnt_rs_launch_count()
    with pytest.raises(pkg.FntRsError) as ei:
        pkg.fnt_rs_encode_noalloc(plan.handle, src, out)
    assert ei.value.code == -9
    assert pkg.fnt_rs_launch_count() == before
    torch.cuda.synchronize()
    assert bool((out == -1).all())
    assert plan.status() == 0


@pytest.mark.parametrize("n,k,n_out,W", [(16384, 8192, 12000, 64), (8192, 4096, 6000, 200)])
def test_noalloc_punctured_within_limit_matches_regular(pkg, n, k, n_out, W):
    plan = pkg.Plan(n, k)
    plan.set_length(n_out)
    assert 0 < pkg.fnt_rs_workspace_bytes(plan.handle, W, pkg.OP_ENCODE) <= pkg.NOALLOC_SCRATCH_BYTES
    for call in range(2):
        src = pkg.to_device(synth.source(77 + call, k, W))
        want = plan.encode(src)  # caller workspace
        got = torch.full((n_out, W), -1, dtype=torch.int32, device="cuda")
        pkg.fnt_rs_encode_noalloc(plan.handle, src, got)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
