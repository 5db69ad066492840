"""Golden fixtures: the paper's printed constants and oracle regression values."""
import os

import numpy as np

import synth

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
P = 65537


def _kv(name):
    out = {}
    for line in open(os.path.join(HERE, name)):
        line = line.split("#")[0].strip()
        if line:
            key, val = line.split()
            out[key] = val
    return out


def test_paper_constants():
    c = _kv("paper_constants.txt")
    p, g, order = int(c["field_prime"]), int(c["primitive_root"]), int(c["order_of_3"])
    assert p == 2 ** 16 + 1 == P
    assert pow(g, order, p) == 1 and pow(g, order // 2, p) != 1
    # Table I / II FNT counts are the cost model the GPU path is compared with
    assert int(c["encode_fnt_count_nonsystematic"]) == 1
    assert int(c["decode_fnt_count_nonsystematic"]) == 8


def test_roots_fixture(oracle_lib):
    for line in open(os.path.join(HERE, "roots.txt")):
        if line.startswith("#"):
            continue
        n, r, rinv, ninv = map(int, line.split())
        assert oracle_lib.root(n) == r
        assert r * rinv % P == 1 and n * ninv % P == 1


def test_example_fixture(oracle_lib):
    rows = [l.split() for l in open(os.path.join(HERE, "example_n16_k8.txt")) if not l.startswith("#")]
    src = [list(map(int, r[1:])) for r in rows if r[0] == "source"]
    enc = [list(map(int, r[1:])) for r in rows if r[0] == "encoded"]
    pos = np.array(list(map(int, [r for r in rows if r[0] == "positions"][0][1:])), dtype=np.uint32)
    s = np.array(src, dtype=np.uint16).T
    assert np.array_equal(s, synth.source(123, 8, 2))
    e = oracle_lib.encode(s, 16)
    assert np.array_equal(e, np.array(enc, dtype=np.uint32).T)
    back, flag = oracle_lib.decode(e[pos], pos, 16, 8)
    assert not flag and np.array_equal(back, s)
