"""Pins for the CPU oracle: facts fixed by the paper and by the mathematics.

Every test here checks the oracle against something other than itself:
number-theoretic facts (Sec. II.A: 3 is a primitive root of GF(65537)),
the DFT written as its defining sum (Sec. II.A), a radix-2 FFT written in
this file, Gaussian elimination on the Vandermonde system (Sec. II.A),
brute-force MDS recovery (Sec. I / II.B), the derivative identity
A_i(x_i) = A'(x_i) (Sec. II.B), the chirp route of step 3 and the power
series of step 5 (Sec. II.B), and closed forms derived from x^n - 1.
"""
import itertools

import numpy as np
import pytest

from oracle import small

P = 65537


def test_three_is_primitive_root():
    # Sec. II.A: 3^65536 = 1 and no smaller power is 1.  The order divides
    # 2^16, so it suffices that 3^(2^15) != 1; it is in fact -1.
    assert pow(3, 65536, P) == 1
    assert pow(3, 32768, P) == P - 1


@pytest.mark.parametrize("log2n", range(1, 17))
def test_root_has_order_n(oracle_lib, log2n):
    n = 1 << log2n
    r = oracle_lib.root(n)
    assert pow(r, n, P) == 1
    assert pow(r, n // 2, P) == P - 1  # exactly order n
    # the code is fixed by this root (Sec. II.B): r_n = r_{2n}^2
    if n < 65536:
        assert pow(oracle_lib.root(2 * n), 2, P) == r


def test_small_roots_are_powers_of_two(oracle_lib):
    # derived: 2 has order 32 mod 65537 (2^16 = -1), so the roots of order
    # <= 32 are powers of two; the GPU butterflies rely on this.
    expect = {2: 16, 4: 24, 8: 12, 16: 6, 32: 19}
    for n, e in expect.items():
        assert oracle_lib.root(n) == pow(2, e, P)


def _fft_radix2(a, r):
    """Recursive radix-2 decimation-in-time FFT over F_p (test-only)."""
    n = len(a)
    if n == 1:
        return list(a)
    even = _fft_radix2(a[0::2], r * r % P)
    odd = _fft_radix2(a[1::2], r * r % P)
    out = [0] * n
    w = 1
    for j in range(n // 2):
        t = w * odd[j] % P
        out[j] = (even[j] + t) % P
        out[j + n // 2] = (even[j] - t) % P
        w = w * r % P
    return out


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64])
def test_c_dft_matches_definition(oracle_lib, n):
    rng = np.random.default_rng(n)
    x = rng.integers(0, P, size=(n, 3), dtype=np.uint32)
    got = oracle_lib.dft(x)
    got_inv = oracle_lib.dft(x, inverse=True)
    r = small.root(n)
    for c in range(3):
        col = [int(v) for v in x[:, c]]
        assert list(got[:, c]) == small.dft_definition(col, r)
        assert list(got_inv[:, c]) == small.dft_definition(col, r, inverse=True)


@pytest.mark.parametrize("n", [128, 256, 1024])
def test_c_dft_matches_fft_and_inverts(oracle_lib, n):
    rng = np.random.default_rng(n)
    x = rng.integers(0, P, size=(n, 2), dtype=np.uint32)
    y = oracle_lib.dft(x)
    r = small.root(n)
    for c in range(2):
        assert list(y[:, c]) == _fft_radix2([int(v) for v in x[:, c]], r)
    assert np.array_equal(oracle_lib.dft(y, inverse=True), x)


@pytest.mark.parametrize("n,k", [(2, 1), (4, 2), (8, 3), (16, 8), (32, 17), (64, 64)])
def test_encode_is_dft_of_zero_padded_source(oracle_lib, n, k):
    # Sec. II.B: encoding applies the FNT to (s_0..s_{k-1}, 0..0).
    rng = np.random.default_rng(7 + n + k)
    s = rng.integers(0, 65536, size=(k, 4), dtype=np.uint16)
    e = oracle_lib.encode(s, n)
    r = small.root(n)
    for c in range(4):
        padded = [int(v) for v in s[:, c]] + [0] * (n - k)
        assert list(e[:, c]) == small.dft_definition(padded, r)


def test_encode_is_linear(oracle_lib):
    rng = np.random.default_rng(3)
    n, k = 256, 100
    a = rng.integers(0, 30000, size=(k, 5), dtype=np.uint16)
    b = rng.integers(0, 30000, size=(k, 5), dtype=np.uint16)
    ea, eb = oracle_lib.encode(a, n), oracle_lib.encode(b, n)
    eab = oracle_lib.encode((a.astype(np.uint32) + b).astype(np.uint16), n)
    assert np.array_equal(eab, (ea.astype(np.uint64) + eb) % P)


def test_mds_brute_force_n8(oracle_lib):
    # Sec. I / II.A: any k of the n symbols recover the source.  Every k and
    # every k-subset of the 8 positions.
    n = 8
    rng = np.random.default_rng(8)
    for k in range(1, n + 1):
        s = rng.integers(0, 65536, size=(k, 3), dtype=np.uint16)
        e = oracle_lib.encode(s, n)
        for subset in itertools.combinations(range(n), k):
            pos = np.array(subset, dtype=np.uint32)
            got, flag = oracle_lib.decode(e[pos], pos, n, k)
            assert not flag
            assert np.array_equal(got, s), (k, subset)


def test_mds_unordered_and_extra_positions(oracle_lib):
    # first k entries of `positions` are used, in the caller's order
    n, k = 16, 6
    rng = np.random.default_rng(16)
    s = rng.integers(0, 65536, size=(k, 4), dtype=np.uint16)
    e = oracle_lib.encode(s, n)
    for _ in range(20):
        pos = rng.permutation(n)[: k + 3].astype(np.uint32)
        got, _ = oracle_lib.decode(e[pos], pos, n, k)
        assert np.array_equal(got, s)


@pytest.mark.parametrize("n,k", [(8, 5), (16, 8), (32, 20), (64, 32)])
def test_lagrange_matches_gaussian_elimination(oracle_lib, n, k):
    # arbitrary received values (not codewords): the interpolant is unique
    rng = np.random.default_rng(n * 100 + k)
    pos = np.sort(rng.choice(n, k, replace=False)).astype(np.uint32)
    v = rng.integers(0, P, size=(k, 3), dtype=np.uint32)
    got, _ = oracle_lib.decode(v, pos, n, k)
    for c in range(3):
        want = small.gauss_decode([int(x) for x in v[:, c]], [int(z) for z in pos], n, k)
        want = [0 if w == 65536 else w for w in want]
        assert list(got[:, c]) == want


@pytest.mark.parametrize("n,k", [(16, 8), (16, 12), (32, 28), (64, 48)])
def test_pattern_derivative_identity_and_closed_form(oracle_lib, n, k):
    rng = np.random.default_rng(n + k)
    pos = np.sort(rng.choice(n, k, replace=False))
    A, dA, w = oracle_lib.pattern(n, k, pos)
    r = small.root(n)
    xs = [pow(r, int(z), P) for z in pos]
    # A(x) = prod (x - x_j): compare with an independent product
    assert list(A) == small.locator(xs)
    erased = sorted(set(range(n)) - set(int(z) for z in pos))
    L = small.locator([pow(r, j, P) for j in erased])
    for i, xi in enumerate(xs):
        # Sec. II.B: A_i(x_i) = prod_{j != i} (x_i - x_j) = A'(x_i)
        prod = 1
        for j, xj in enumerate(xs):
            if j != i:
                prod = prod * (xi - xj) % P
        assert int(dA[i]) == prod
        assert int(w[i]) * prod % P == 1
        # derived from x^n - 1 = A(x) L(x): A'(x_i) = n / (x_i L(x_i))
        assert int(dA[i]) == n * small.inv(xi * small.poly_eval(L, xi)) % P


@pytest.mark.parametrize("n,k", [(8, 4), (16, 12), (32, 28)])
def test_chirp_step3_matches_direct_evaluation(oracle_lib, n, k):
    # Sec. II.B step 3 (corrected reading): chirp route == evaluation == DFT
    rng = np.random.default_rng(k)
    pos = np.sort(rng.choice(n, k, replace=False))
    A, dA, _ = oracle_lib.pattern(n, k, pos)
    dcoef = small.derivative([int(a) for a in A])
    chirp = small.chirp_eval(dcoef, n)
    r = small.root(n)
    direct = [small.poly_eval(dcoef, pow(r, i, P)) for i in range(n)]
    assert chirp == direct
    col = np.array(dcoef + [0] * (n - len(dcoef)), dtype=np.uint32).reshape(n, 1)
    assert list(oracle_lib.dft(col)[:, 0]) == direct
    assert [direct[int(z)] for z in pos] == [int(v) for v in dA]


@pytest.mark.parametrize("n,k", [(8, 4), (16, 8), (16, 12), (32, 28), (64, 48)])
def test_series_route_matches_lagrange_and_zero_tail(oracle_lib, n, k):
    # Sec. II.B steps 4-6 written literally; coefficients k..n-1 of (A S)
    # mod x^n vanish because P = A S has degree < k.
    rng = np.random.default_rng(n * k)
    pos = np.sort(rng.choice(n, k, replace=False)).astype(np.uint32)
    v = rng.integers(0, P, size=(k, 2), dtype=np.uint32)
    got, _ = oracle_lib.decode(v, pos, n, k)
    for c in range(2):
        coeffs, prod = small.series_decode([int(x) for x in v[:, c]], [int(z) for z in pos], n, k)
        assert list(got[:, c]) == [0 if x == 65536 else x for x in coeffs]
        assert all(x == 0 for x in prod[k:n])


def test_lossless_decode_is_inverse_dft(oracle_lib):
    # Sec. II.B: with nothing lost, decoding is the inverse FNT's first k.
    n, k = 64, 40
    rng = np.random.default_rng(64)
    s = rng.integers(0, 65536, size=(k, 3), dtype=np.uint16)
    e = oracle_lib.encode(s, n)
    back = oracle_lib.dft(e, inverse=True)
    assert np.array_equal(back[:k], s.astype(np.uint32))
    assert not back[k:].any()
    got, _ = oracle_lib.decode(e, np.arange(n, dtype=np.uint32), n, k)
    assert np.array_equal(got, s)


def test_range_flag_when_coefficient_is_65536(oracle_lib):
    # a "source" whose first coefficient is the field element 65536 cannot be
    # a 16-bit symbol: the decoder writes 0 and raises the flag.
    n, k = 16, 8
    coeffs = [65536, 5, 6, 7, 8, 9, 10, 11]
    r = small.root(n)
    e = [small.poly_eval(coeffs, pow(r, j, P)) for j in range(n)]
    pos = np.arange(3, 3 + k, dtype=np.uint32)
    v = np.array([[e[int(z)]] for z in pos], dtype=np.uint32)
    got, flag = oracle_lib.decode(v, pos, n, k)
    assert flag
    assert list(got[:, 0]) == [0, 5, 6, 7, 8, 9, 10, 11]


def test_bad_positions_rejected(oracle_lib):
    n, k = 16, 4
    v = np.zeros((4, 1), dtype=np.uint32)
    with pytest.raises(ValueError):
        oracle_lib.decode(v, np.array([0, 1, 1, 2], dtype=np.uint32), n, k)  # duplicate
    with pytest.raises(ValueError):
        oracle_lib.decode(v, np.array([0, 1, 2, 16], dtype=np.uint32), n, k)  # out of range
    with pytest.raises(ValueError):
        oracle_lib.decode(v[:3], np.array([0, 1, 2], dtype=np.uint32), n, k)  # fewer than k


def test_encode_rows_matches_definition(oracle_lib):
    n, k = 64, 20
    rng = np.random.default_rng(5)
    s = rng.integers(0, 65536, size=(k, 3), dtype=np.uint16)
    rows = np.array([0, 5, 63, 17], dtype=np.uint32)
    got = oracle_lib.encode_rows(s, n, rows)
    r = small.root(n)
    for c in range(3):
        full = small.dft_definition([int(v) for v in s[:, c]] + [0] * (n - k), r)
        assert list(got[:, c]) == [full[j] for j in rows]
