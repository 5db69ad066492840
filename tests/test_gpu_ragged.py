"""Ragged batches: groups of mixed (n, k, W, erasure pattern) in one graph launch.

Each group must round-trip exactly (decode(encode(s)) == s on every codeword),
match the oracle on sampled columns, and give the same bits as the plain
per-group calls and as a plan used on its own (the same alone and in the mix).
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


def _groups(pkg, seed, ngroups, log2n=(6, 16), log2w=(2, 6)):
    specs = synth.ragged_groups(seed=seed, groups=ngroups, log2n=log2n, log2bytes=log2w)
    groups = []
    for i, g in enumerate(specs):
        n, k, W = g["n"], g["k"], g["W"]
        src = synth.source(g["seed"], k, W)
        d = {"n": n, "k": k, "src_h": src, "src": pkg.to_device(src),
             "enc": torch.zeros((n, W), dtype=torch.int32, device="cuda"),
             "out": torch.zeros((k, W), dtype=torch.int16, device="cuda"),
             "positions": g["positions"] if i % 5 != 4 else None}  # some encode-only groups
        groups.append(d)
    return groups


def test_ragged_graph_round_trip_and_oracle(pkg):
    groups = _groups(pkg, seed=41, ngroups=36)
    r = pkg.fnt_rs_ragged_create(groups, nstreams=6)
    try:
        info = pkg.fnt_rs_ragged_info(r)
        assert info["groups"] == 36
        # every code with n >= 256 runs in the persistent kernel, shorter ones per group
        assert info["persistent_groups"] == sum(g["n"] >= 256 for g in groups)
        assert 0 < info["persistent_groups"] < 36
        for g in groups:  # creation already ran the batch once; clear and rerun by graph
            g["enc"].zero_()
            g["out"].zero_()
        pkg.fnt_rs_ragged_run(r)
        torch.cuda.synchronize()
        assert pkg.fnt_rs_ragged_status(r) == 0
        rng = np.random.default_rng(5)
        for g in groups:
            n, k = g["n"], g["k"]
            enc = pkg.to_host(g["enc"])
            W = enc.shape[1]
            c = int(rng.integers(0, W))
            want = oracle.encode(np.ascontiguousarray(g["src_h"][:, [c]]), n)
            assert np.array_equal(enc[:, [c]], want), (n, k)
            if g["positions"] is not None:
                assert np.array_equal(pkg.to_host(g["out"]), g["src_h"]), (n, k)
    finally:
        pkg.fnt_rs_ragged_destroy(r)


def test_ragged_same_alone_and_in_mix(pkg):
    groups = _groups(pkg, seed=43, ngroups=20, log2n=(8, 14))
    r = pkg.fnt_rs_ragged_create(groups, nstreams=4)
    try:
        pkg.fnt_rs_ragged_run(r)
        torch.cuda.synchronize()
        mix_enc = [pkg.to_host(g["enc"]) for g in groups]
        mix_out = [pkg.to_host(g["out"]) for g in groups]
        for g in groups:
            g["enc"].zero_()
            g["out"].zero_()
        pkg.fnt_rs_ragged_run_plain(r)
        torch.cuda.synchronize()
        for i, g in enumerate(groups):
            assert np.array_equal(pkg.to_host(g["enc"]), mix_enc[i])
            assert np.array_equal(pkg.to_host(g["out"]), mix_out[i])
            plan = pkg.Plan(g["n"], g["k"])  # the group on its own
            assert np.array_equal(pkg.to_host(plan.encode(g["src"])), mix_enc[i])
            if g["positions"] is not None:
                alone = plan.decode_slots(pkg.to_device(mix_enc[i]), g["positions"])
                assert np.array_equal(pkg.to_host(alone), mix_out[i])
    finally:
        pkg.fnt_rs_ragged_destroy(r)


def test_ragged_persistent_kernel_groups(pkg):
    # only tile-sized codes (256 <= n <= 8192, every rate): the whole batch runs
    # in the persistent kernel; 48 groups over 6 lengths and 4 rates means many
    # groups share a plan, so their pattern builds run side by side in one launch
    groups = _groups(pkg, seed=47, ngroups=48, log2n=(8, 13), log2w=(2, 8))
    r = pkg.fnt_rs_ragged_create(groups, nstreams=4)
    try:
        info = pkg.fnt_rs_ragged_info(r)
        assert info["persistent_groups"] == 48
        assert info["persistent_items"] > 48
        rng = np.random.default_rng(9)
        first = None
        for rep in range(3):  # the graph's counters start from zero on every run
            for g in groups:
                g["enc"].zero_()
                g["out"].zero_()
            pkg.fnt_rs_ragged_run(r)
            torch.cuda.synchronize()
            assert pkg.fnt_rs_ragged_status(r) == 0
            got = [(pkg.to_host(g["enc"]), pkg.to_host(g["out"])) for g in groups]
            if first is None:
                first = got
            for i, g in enumerate(groups):
                assert np.array_equal(got[i][0], first[i][0]) and np.array_equal(got[i][1],
                                                                                  first[i][1])
                if g["positions"] is not None:
                    assert np.array_equal(got[i][1], g["src_h"]), (g["n"], g["k"])
        for i, g in enumerate(groups):
            n = g["n"]
            c = int(rng.integers(0, g["src_h"].shape[1]))
            want = oracle.encode(np.ascontiguousarray(g["src_h"][:, [c]]), n)
            assert np.array_equal(first[i][0][:, [c]], want), (n, g["k"])
        # per-group plain launches give the same bits
        for g in groups:
            g["enc"].zero_()
            g["out"].zero_()
        pkg.fnt_rs_ragged_run_plain(r)
        torch.cuda.synchronize()
        for i, g in enumerate(groups):
            assert np.array_equal(pkg.to_host(g["enc"]), first[i][0])
            assert np.array_equal(pkg.to_host(g["out"]), first[i][1])
    finally:
        pkg.fnt_rs_ragged_destroy(r)


def test_ragged_long_codes_in_one_persistent_launch(pkg):
    # every long length at every rate of the ragged batch: one-CTA tiles for
    # n = 16384 and for n = 32768 at rate 1/2, split transforms run inside one
    # CTA per 8-column item for n = 65536 and for n = 32768 above rate 1/2, and
    # the long pattern builds (spectrum item + digit items) for n >= 32768;
    # widths that are not multiples of the item width, some encode-only groups,
    # and a few short codes in the same launch
    shapes = [(16384, 8192, 9), (16384, 12288, 5), (16384, 14336, 4), (32768, 16384, 3),
              (32768, 21845, 11), (32768, 28672, 8), (65536, 32768, 13), (65536, 43690, 6),
              (65536, 49152, 17), (65536, 57344, 4), (4096, 3072, 20), (256, 128, 40),
              (65536, 32768, 10), (32768, 24576, 9)]
    groups = []
    for i, (n, k, W) in enumerate(shapes):
        src = synth.source(700 + i, k, W)
        pos = synth.received_positions(n, synth.erased_uniform(800 + i, n, k))
        groups.append({"n": n, "k": k, "src_h": src, "src": pkg.to_device(src),
                       "enc": torch.zeros((n, W), dtype=torch.int32, device="cuda"),
                       "out": torch.zeros((k, W), dtype=torch.int16, device="cuda"),
                       "positions": pos if i not in (3, 12) else None})
    r = pkg.fnt_rs_ragged_create(groups, nstreams=2)
    try:
        info = pkg.fnt_rs_ragged_info(r)
        assert info["persistent_groups"] == len(groups)
        rng = np.random.default_rng(13)
        first = None
        for rep in range(2):
            for g in groups:
                g["enc"].zero_()
                g["out"].zero_()
            pkg.fnt_rs_ragged_run(r)
            torch.cuda.synchronize()
            assert pkg.fnt_rs_ragged_status(r) == 0
            got = [(pkg.to_host(g["enc"]), pkg.to_host(g["out"])) for g in groups]
            if first is None:
                first = got
            for i, g in enumerate(groups):
                assert np.array_equal(got[i][0], first[i][0]), shapes[i]
                assert np.array_equal(got[i][1], first[i][1]), shapes[i]
                if g["positions"] is not None:
                    assert np.array_equal(got[i][1], g["src_h"]), shapes[i]
        for i, g in enumerate(groups):  # encoded rows by Horner (O(k) each)
            n, k = g["n"], g["k"]
            W = g["src_h"].shape[1]
            cols = [0, W - 1]
            rows = np.sort(rng.choice(n, 3, replace=False)).astype(np.uint32)
            want = oracle.encode_rows(np.ascontiguousarray(g["src_h"][:, cols]), n, rows)
            assert np.array_equal(first[i][0][rows][:, cols], want), shapes[i]
        # per-group plain launches give the same bits
        for g in groups:
            g["enc"].zero_()
            g["out"].zero_()
        pkg.fnt_rs_ragged_run_plain(r)
        torch.cuda.synchronize()
        for i, g in enumerate(groups):
            assert np.array_equal(pkg.to_host(g["enc"]), first[i][0]), shapes[i]
            assert np.array_equal(pkg.to_host(g["out"]), first[i][1]), shapes[i]
    finally:
        pkg.fnt_rs_ragged_destroy(r)
