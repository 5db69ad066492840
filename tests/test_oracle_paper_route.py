"""Pins of the paper's decode route as the GPU schedule FNT_RS_SCHED_PAPER runs it.

Sec. II.B evaluates on geometric progressions with the chirp identity
r^(ij) = b_(i+j) / (b_i b_j), b_i = r^(i(i-1)/2), which makes an evaluation the
middle coefficients of one product; Sec. III computes the products of steps 5
and 6 with transforms of length 2n.  Here the whole route is written in pure
Python with the DFT of Sec. II.A taken by its definition, and checked against
Gaussian elimination on the Vandermonde system (a route that shares nothing
with it): step 3 by the chirp, step 5 as a cyclic product of length 2n whose
wrapped terms fall below the coefficients read, step 6 as a cyclic product of
length 2n.  A planted mistake in each step must break the agreement.
"""
import numpy as np
import pytest

from oracle import small

P = 65537


def cyclic(a, b, m, w):
    """Cyclic product of length m by DFTs of root w (order m), by definition."""
    fa = small.dft_definition(list(a) + [0] * (m - len(a)), w)
    fb = small.dft_definition(list(b) + [0] * (m - len(b)), w)
    return small.dft_definition([x * y % P for x, y in zip(fa, fb)], w, inverse=True)


def chirp_b(q, count):
    return [pow(q, i * (i - 1) // 2, P) for i in range(count)]


def paper_route(values, positions, n, k, mistake=None):
    r = small.root(n)
    w2 = small.root(2 * n)  # root of order 2n for the length-2n products
    z = list(positions[:k])
    xs = [pow(r, zi, P) for zi in z]
    A = small.locator(xs)  # step 1
    dA = small.derivative(A)  # step 2
    # step 3: A'(r^i) = b_i^-1 sum_j (a'_j / b_j) b_(i+j), middle coefficients n-1+i
    b = chirp_b(r, 2 * n)
    c = [dA[j] * small.inv(b[j]) % P if j < len(dA) else 0 for j in range(n)]
    G = [c[n - 1 - t] for t in range(n)]
    Y = cyclic(G, b, 2 * n, w2)
    off = n - 1 if mistake != "step3_offset" else n
    dAv = [Y[off + zi] * small.inv(b[zi]) % P for zi in z]
    # step 4
    ns = [values[i] * small.inv(dAv[i]) % P for i in range(k)]
    # step 5: N'(q^m) = b'_m^-1 sum_z (n_z / b'_z) b'_(m+z), q = r^-1; S_j = -N'(q^(j+1))
    q = small.inv(r)
    bq = chirp_b(q, 2 * n)
    g = [0] * n
    for i, zi in enumerate(z):
        g[n - 1 - zi] = ns[i] * small.inv(bq[zi]) % P
    Y = cyclic(g, bq, 2 * n, w2)
    shift = 1 if mistake != "step5_shift" else 0
    S = [(-Y[n - 1 + j + shift] * small.inv(bq[j + shift])) % P for j in range(k)]
    if mistake == "step5_sign":
        S = [(-s) % P for s in S]
    # step 6: P = (A S) mod x^k
    Am = A[:k] if mistake != "step6_full_A" else A
    prod = cyclic(Am, S, 2 * n, w2)
    return [prod[j] for j in range(k)]


@pytest.mark.parametrize("n,k", [(8, 3), (16, 8), (16, 5), (32, 16), (32, 9)])
def test_paper_route_matches_gauss(n, k):
    rng = np.random.default_rng(n * 7 + k)
    for _ in range(3):
        pos = [int(x) for x in rng.permutation(n)[:k]]
        vals = [int(x) for x in rng.integers(0, P, k)]
        assert paper_route(vals, pos, n, k) == small.gauss_decode(vals, pos, n, k)


def test_chirp_identity_and_recurrence():
    # b_(i+1) = r^i b_i (the printed "q^i" read as r^i) and r^(ij) = b_(i+j) / (b_i b_j)
    n = 16
    r = small.root(n)
    b = chirp_b(r, 2 * n)
    for i in range(2 * n - 1):
        assert b[i + 1] == pow(r, i, P) * b[i] % P
    for i in range(n):
        for j in range(n):
            assert pow(r, i * j, P) == b[i + j] * small.inv(b[i] * b[j] % P) % P


@pytest.mark.parametrize("mistake", ["step3_offset", "step5_shift", "step5_sign", "step6_full_A"])
def test_planted_mistakes_break_the_route(mistake):
    n, k = 16, 7
    rng = np.random.default_rng(3)
    pos = [int(x) for x in rng.permutation(n)[:k]]
    vals = [int(x) for x in rng.integers(0, P, k)]
    good = small.gauss_decode(vals, pos, n, k)
    bad = paper_route(vals, pos, n, k, mistake)
    if mistake == "step6_full_A":
        # the x^k term of A only reaches coefficients >= k: harmless, as the route relies on
        assert bad == good
    else:
        assert bad != good
