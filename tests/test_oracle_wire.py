"""Pins of the oracle's 16-bit wire format (Sec. II.B, "Design of the code on
GF(65537)": symbols travel as 16 bits, the positions of the value 65536 go
in the packet headers).

The pins do not reuse the oracle's code: codewords whose symbol 65536 is
known in closed form (k = 2, source (1, 65535): e_j = 1 - 2 r^j, so e_0 = -1),
explicit-power evaluation (oracle.small), numpy's own comparison for the
escape set, and the decode of wire packets against the source.
"""
import numpy as np
import pytest

import oracle
from oracle import small, wire

P = 65537


def test_closed_form_escape_k2():
    # s(x) = 1 + 65535 x = 1 - 2x: s(r^0) = -1 = 65536, s(r^(n/2)) = 1 + 2 = 3
    n, k, W = 16, 2, 5
    src = np.zeros((k, W), dtype=np.uint16)
    src[0, :] = 1
    src[1, :] = 65535
    src[:, 3] = (7, 9)  # one ordinary column: 7 + 9 r^j never equals -1 here
    enc = oracle.encode(src, n)
    r = small.root(n)
    for j in range(n):
        assert enc[j, 0] == small.poly_eval([1, 65535], pow(r, j, P))
    assert enc[0, 0] == 65536 and enc[n // 2, 0] == 3
    sym, esc = wire.to_wire(enc)
    want = sorted((int(j), int(c)) for j in range(n) for c in range(W) if enc[j, c] == 65536)
    assert [tuple(e) for e in esc] == want
    assert (0, 0) in want and all(c != 3 for _, c in want)
    assert sym[0, 0] == 0 and sym.dtype == np.uint16
    assert np.array_equal(wire.from_wire(sym, esc), enc)


def test_low_bits_and_escape_set():
    rng = np.random.default_rng(4)
    enc = rng.integers(0, P, (40, 33), dtype=np.uint32)
    hits = rng.choice(enc.size, 25, replace=False)
    enc.reshape(-1)[hits] = 65536
    sym, esc = wire.to_wire(enc)
    assert np.array_equal(sym, (enc & 0xFFFF).astype(np.uint16))  # 65536 -> 0, others kept
    rows, cols = np.nonzero(enc == 65536)
    assert np.array_equal(esc, np.stack([rows, cols], 1).astype(np.uint32))
    assert len(esc) == 25
    assert np.array_equal(wire.from_wire(sym, esc), enc)


def test_from_wire_rejects_inconsistent_input():
    sym = np.zeros((2, 3), dtype=np.uint16)
    sym[1, 2] = 5
    with pytest.raises(ValueError):
        wire.from_wire(sym, np.array([[1, 2]], dtype=np.uint32))  # escaped symbol sent as 5
    with pytest.raises(ValueError):
        wire.from_wire(sym, np.array([[2, 0]], dtype=np.uint32))  # no packet 2
    with pytest.raises(ValueError):
        wire.to_wire(np.array([[65537]], dtype=np.uint32))


def test_select_rows_renumbers():
    esc = np.array([[0, 1], [3, 0], [3, 4], [5, 2]], dtype=np.uint32)
    got = wire.select_rows(esc, [5, 3, 2])
    assert [tuple(e) for e in got] == [(0, 2), (1, 0), (1, 4)]


@pytest.mark.parametrize("n,k,W", [(16, 2, 64), (64, 20, 40), (512, 256, 24)])
def test_decode_from_wire_packets(n, k, W):
    rng = np.random.default_rng(n + k)
    src = rng.integers(0, 65536, (k, W), dtype=np.uint16)
    if k == 2:
        src[:, : W // 2] = np.array([[1], [65535]], dtype=np.uint16)  # e_0 = 65536
    enc = oracle.encode(src, n)
    sym, esc = wire.to_wire(enc)
    pos = rng.permutation(n)[:k].astype(np.uint32)
    if k == 2:
        pos = np.array([0, 1 + rng.integers(0, n - 1)], dtype=np.uint32)  # packet 0 has escapes
    rsym = sym[pos]
    resc = wire.select_rows(esc, pos)
    assert len(resc) == int((enc[pos] == 65536).sum())
    out, flag = oracle.decode(wire.from_wire(rsym, resc), pos, n, k)
    assert not flag and np.array_equal(out, src)
    # the escape list is what makes this work: without it the decode is wrong
    if len(resc):
        bad, _ = oracle.decode(rsym.astype(np.uint32), pos, n, k)
        assert not np.array_equal(bad, src)
