"""Failure detection on the GPU without a fault: a stalled producer.

The ragged persistent kernel makes a decode item wait (bounded) until its
group's encode tiles and pattern build are done.  FNTRS_TEST_STALL_GROUP=g
makes group g's decode items wait for one encode tile more than exists, a
producer that never finishes: the waits must give up after their bound, set
FNT_RS_E_TIMEOUT in the status word the host reads, skip that group's decode,
let every other group finish correctly, and leave the context usable.
"""
import time

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


def _group(pkg, n, k, W, seed):
    src = synth.source(seed, k, W)
    return {"n": n, "k": k, "src_h": src, "src": pkg.to_device(src),
            "enc": torch.zeros((n, W), dtype=torch.int32, device="cuda"),
            "out": torch.zeros((k, W), dtype=torch.int16, device="cuda"),
            "positions": synth.received_positions(n, synth.erased_uniform(seed + 1, n, k))}


def test_stalled_producer_times_out_and_the_rest_completes(pkg, monkeypatch):
    groups = [_group(pkg, 256, 128, 32, 1), _group(pkg, 512, 200, 24, 3),
              _group(pkg, 1024, 512, 16, 5)]
    monkeypatch.setenv("FNTRS_TEST_STALL_GROUP", "1")
    t0 = time.perf_counter()
    r = pkg.fnt_rs_ragged_create(groups, nstreams=2)  # runs the batch once
    try:
        torch.cuda.synchronize()
        waited = time.perf_counter() - t0
        assert pkg.fnt_rs_ragged_info(r)["persistent_groups"] == 3
        assert pkg.fnt_rs_ragged_status(r) == pkg.E_TIMEOUT
        for i, g in enumerate(groups):
            enc = pkg.to_host(g["enc"])
            assert np.array_equal(enc, oracle.encode(g["src_h"], g["n"])), i  # producers ran
            if i != 1:
                assert np.array_equal(pkg.to_host(g["out"]), g["src_h"]), i
        # the graph replays the same way: the stall is reported again, the rest is right
        for g in groups:
            g["out"].zero_()
        pkg.fnt_rs_ragged_run(r)
        torch.cuda.synchronize()
        assert pkg.fnt_rs_ragged_status(r) == pkg.E_TIMEOUT
        assert np.array_equal(pkg.to_host(groups[2]["out"]), groups[2]["src_h"])
    finally:
        pkg.fnt_rs_ragged_destroy(r)
    assert waited < 120, waited
    # the context is still usable: a fresh batch without the stall and a plain round trip
    monkeypatch.delenv("FNTRS_TEST_STALL_GROUP")
    groups = [_group(pkg, 256, 128, 32, 7)]
    r = pkg.fnt_rs_ragged_create(groups, nstreams=1)
    try:
        torch.cuda.synchronize()
        assert pkg.fnt_rs_ragged_status(r) == 0
        assert np.array_equal(pkg.to_host(groups[0]["out"]), groups[0]["src_h"])
    finally:
        pkg.fnt_rs_ragged_destroy(r)
    plan = pkg.Plan(512, 256)
    src = synth.source(9, 256, 8)
    enc = pkg.to_host(plan.encode(pkg.to_device(src)))
    pos = synth.received_positions(512, synth.erased_uniform(10, 512, 256))
    out = pkg.to_host(plan.decode(pkg.to_device(np.ascontiguousarray(enc[pos])), pos))
    assert np.array_equal(out, src) and plan.status() == 0
    print(f"stalled decode items gave up after {waited:.2f} s")
