"""Pure-Python restatements for tiny cases (n <= 64).

TEST INFRASTRUCTURE ONLY.  Each routine computes a quantity of the paper by a
route different from the C oracle, so that the two can pin each other:

* :func:`dft_definition`   -- DFT / inverse DFT written as the sums of Sec. II.A;
* :func:`gauss_decode`     -- solve the k x k Vandermonde system of Sec. II.A
                              (the FNT matrix's rows, restricted to the received
                              points) by Gaussian elimination mod p;
* :func:`chirp_eval`       -- step 3 of the interpolation by the chirp / product
                              route of Sec. II.B, in the corrected reading
                              (b_{i+1} = r^i b_i, c_j = a'_j / b_j);
* :func:`series_decode`    -- steps 4-6 of Sec. II.B: n_i = v_i / A'(x_i),
                              S(x) = -sum_j N'(r^(-j-1)) x^j, P = (A S) mod x^k.
"""
from __future__ import annotations

P = 65537


def inv(a: int) -> int:
    a %= P
    if a == 0:
        raise ZeroDivisionError("0 has no inverse mod p")
    return pow(a, P - 2, P)


def root(n: int) -> int:
    """3 has order 2^16 (Sec. II.A), so 3^(65536/n) has order n (Sec. II.B)."""
    assert n >= 1 and n & (n - 1) == 0 and n <= 65536
    return pow(3, 65536 // n, P)


def dft_definition(a, r: int, inverse: bool = False):
    """A_j = sum_i a_i r^(ij); the inverse uses r^-1 and the factor n^-1."""
    n = len(a)
    if inverse:
        r = inv(r)
    out = []
    for j in range(n):
        acc = 0
        for i in range(n):
            acc += a[i] * pow(r, i * j, P)
        acc %= P
        if inverse:
            acc = acc * inv(n) % P
        out.append(acc)
    return out


def poly_eval(coeffs, x: int) -> int:
    """sum_i c_i x^i with explicit powers (not Horner)."""
    return sum(c * pow(x, i, P) for i, c in enumerate(coeffs)) % P


def gauss_decode(values, positions, n: int, k: int):
    """Recover s from s(r^(z_i)) = v_i, i < k, by Gaussian elimination mod p.

    The system is the k x k matrix M[i][j] = (r^(z_i))^j of Sec. II.A's
    Vandermonde view of the FNT.
    """
    r = root(n)
    rows = []
    for i in range(k):
        x = pow(r, positions[i], P)
        rows.append([pow(x, j, P) for j in range(k)] + [values[i] % P])
    for col in range(k):
        piv = next(i for i in range(col, k) if rows[i][col] % P)
        rows[col], rows[piv] = rows[piv], rows[col]
        f = inv(rows[col][col])
        rows[col] = [v * f % P for v in rows[col]]
        for i in range(k):
            if i != col and rows[i][col]:
                g = rows[i][col]
                rows[i] = [(a - g * b) % P for a, b in zip(rows[i], rows[col])]
    return [rows[i][k] for i in range(k)]


def poly_mul(a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] = (out[i + j] + x * y) % P
    return out


def locator(points):
    """A(x) = prod_j (x - x_j), coefficients low to high."""
    A = [1]
    for x in points:
        A = poly_mul(A, [(-x) % P, 1])
    return A


def derivative(a):
    return [(i * a[i]) % P for i in range(1, len(a))]


def chirp_eval(coeffs, n: int):
    """Evaluate a polynomial of degree < n at r^i, i < n, by the chirp route.

    t_i = i(i-1)/2, b_i = r^(t_i) for i <= 2n-2, c_j = a_j / b_j, and
    A(r^i) = b_i^-1 sum_j c_j b_(i+j): the sum is read off the coefficients
    n-1 .. 2n-2 of (sum_j c_j x^(n-1-j)) * (sum_i b_i x^i).
    """
    r = root(n)
    a = list(coeffs) + [0] * (n - len(coeffs))
    b = [pow(r, i * (i - 1) // 2, P) for i in range(2 * n - 1)]
    c = [a[j] * inv(b[j]) % P for j in range(n)]
    rev_c = [c[n - 1 - i] for i in range(n)]
    prod = poly_mul(rev_c, b)
    return [prod[n - 1 + i] * inv(b[i]) % P for i in range(n)]


def series_decode(values, positions, n: int, k: int):
    """Steps 1-6 of the interpolation algorithm of Sec. II.B, literally.

    x_i = r^(z_i); A = prod (x - x_i); n_i = v_i / A'(x_i);
    S(x) = sum_i n_i / (x - x_i) mod x^n = -sum_j N'(r^(-j-1)) x^j with
    N'(y) = sum_i n_i y^(z_i); P = A * S truncated to degree < k.
    """
    r = root(n)
    z = list(positions[:k])
    xs = [pow(r, zi, P) for zi in z]
    A = locator(xs)
    dA = derivative(A)
    ns = [values[i] * inv(poly_eval(dA, xs[i])) % P for i in range(k)]
    rinv = inv(r)
    S = []
    for j in range(n):
        y = pow(rinv, j + 1, P)
        S.append((-sum(ns[i] * pow(y, z[i], P) for i in range(k))) % P)
    prod = poly_mul(A, S)
    return [prod[j] for j in range(k)], prod
