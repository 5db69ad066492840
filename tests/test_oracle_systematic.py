"""Pins of the oracle's systematic code, puncturing and full-field interpolation.

The systematic construction ("Toward a systematic code"): the intermediate
symbols are the interpolant of the k source values at r^0..r^(k-1), and the
codeword holds that polynomial's values at r^j; decoding interpolates the first
k received points and evaluates at r^0..r^(k-1).  Puncturing keeps the first
n_out < n positions (the non-power-of-two case of Sec. II.B).

The pins do not reuse the oracle's arithmetic: Gaussian elimination on the
Vandermonde system and explicit-power evaluation (oracle.small), the
systematic property itself, MDS recovery from every k-subset, and planted
mistakes in the C source that these facts must catch.
"""
import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import small

P = 65537
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "fnt_rs_oracle.c")


def _gauss_codeword(src_col, n, k, n_out):
    """Values at r^j (j < n_out) of the interpolant of src at r^0..r^(k-1), in pure Python."""
    coef = small.gauss_decode([int(v) for v in src_col], list(range(k)), n, k)
    r = small.root(n)
    return [small.poly_eval(coef, pow(r, j, P)) for j in range(n_out)]


@pytest.mark.parametrize("n,k", [(8, 4), (16, 5), (16, 16), (32, 7)])
def test_systematic_encode_matches_gauss(n, k):
    rng = np.random.default_rng(n + k)
    src = rng.integers(0, 65536, (k, 3), dtype=np.uint16)
    enc = oracle.encode_sys(src, n)
    assert np.array_equal(enc[:k], src.astype(np.uint32))  # the systematic rows
    for c in range(3):
        assert list(enc[:, c]) == _gauss_codeword(src[:, c], n, k, n)


@pytest.mark.parametrize("n,k", [(64, 20), (512, 256), (4096, 3000)])
def test_systematic_rows_and_round_trip(n, k):
    rng = np.random.default_rng(k)
    src = rng.integers(0, 65536, (k, 4), dtype=np.uint16)
    enc = oracle.encode_sys(src, n)
    assert np.array_equal(enc[:k], src.astype(np.uint32))
    pos = rng.permutation(n)[:k]
    out, flag = oracle.decode_sys(enc[pos], pos, n, k)
    assert not flag and np.array_equal(out, src)
    # the codeword is one polynomial of degree < k: any k points give the same interpolant
    pos2 = rng.permutation(n)[:k]
    assert np.array_equal(oracle.interpolate(enc[pos], pos, n, k),
                          oracle.interpolate(enc[pos2], pos2, n, k))


def test_systematic_every_k_subset_n8():
    n, k = 8, 4
    rng = np.random.default_rng(3)
    src = rng.integers(0, 65536, (k, 2), dtype=np.uint16)
    enc = oracle.encode_sys(src, n)
    for pos in itertools.combinations(range(n), k):
        pos = np.array(pos, dtype=np.uint32)
        out, flag = oracle.decode_sys(enc[pos], pos, n, k)
        assert not flag and np.array_equal(out, src), pos


def test_interpolate_matches_gauss_on_arbitrary_values():
    n, k = 16, 6
    rng = np.random.default_rng(5)
    pos = np.array([2, 3, 7, 8, 11, 14], dtype=np.uint32)
    v = rng.integers(0, P, (k, 4), dtype=np.uint32)
    got = oracle.interpolate(v, pos, n, k)
    for c in range(4):
        assert list(got[:, c]) == small.gauss_decode([int(t) for t in v[:, c]],
                                                     [int(z) for z in pos], n, k)
    # decode_sys = that interpolant's values at r^0..r^(k-1); 65536 -> 0 and the flag
    out, flag = oracle.decode_sys(v, pos, n, k)
    r = small.root(n)
    saw = False
    for c in range(4):
        coef = small.gauss_decode([int(t) for t in v[:, c]], [int(z) for z in pos], n, k)
        vals = [small.poly_eval(coef, pow(r, j, P)) for j in range(k)]
        saw = saw or 65536 in vals
        assert list(out[:, c]) == [0 if x == 65536 else x for x in vals]
    assert flag == saw


def test_interpolate_keeps_65536():
    # a received word whose interpolant has the coefficient 65536 = -1: v = -1 at every point
    n, k = 8, 3
    pos = np.array([0, 3, 6], dtype=np.uint32)
    v = np.full((k, 1), P - 1, dtype=np.uint32)
    coef = oracle.interpolate(v, pos, n, k)
    assert list(coef[:, 0]) == [P - 1, 0, 0]  # the constant polynomial -1
    out, flag = oracle.decode(v, pos, n, k)
    assert flag and list(out[:, 0]) == [0, 0, 0]


@pytest.mark.parametrize("n,k,n_out", [(16, 5, 11), (64, 20, 33), (512, 100, 300)])
def test_puncturing_keeps_a_prefix(n, k, n_out):
    rng = np.random.default_rng(n_out)
    src = rng.integers(0, 65536, (k, 3), dtype=np.uint16)
    full = oracle.encode_sys(src, n)
    assert np.array_equal(oracle.encode_sys(src, n, n_out), full[:n_out])
    # any k of the n_out kept positions still recover the source (MDS)
    pos = rng.permutation(n_out)[:k]
    out, flag = oracle.decode_sys(full[pos], pos, n, k)
    assert not flag and np.array_equal(out, src)


# ------------------------------------------------------------ planted mistakes
MUTANTS = {
    # interpolation points shifted by one position
    "sys_points_shifted": ("for (uint32_t i = 0; i < k; ++i) pos[i] = i;",
                           "for (uint32_t i = 0; i < k; ++i) pos[i] = i + 1;"),
    # evaluation with the coefficients reversed
    "eval_reversed": ("acc = orc_add(orc_mul(acc, x), coef[(size_t)i * ld_coef + c]);",
                      "acc = orc_add(orc_mul(acc, x), coef[(size_t)(k - 1 - i) * ld_coef + c]);"),
    # Lagrange weight 1/A'(x_i) dropped
    "interp_no_weight": ("uint32_t cf = orc_mul(recv[(size_t)i * ld_recv + c] % ORC_P, w[i]);",
                         "uint32_t cf = recv[(size_t)i * ld_recv + c] % ORC_P;"),
    # systematic decode evaluating at the inverse root
    "decode_sys_inverse_root": ("eval_rows(r, k, coef, W, k, vals, W, W, nthreads);",
                                "eval_rows(orc_inv(r), k, coef, W, k, vals, W, W, nthreads);"),
}


def _lib(path_c, so):
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(path_c), "-o",
                           str(so)])
    lib = ctypes.CDLL(str(so))
    u32, sz, i32, vp = ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p
    lib.orc_encode_sys.argtypes = [u32, u32, u32, vp, sz, u32, vp, sz, sz, i32]
    lib.orc_decode_sys.argtypes = [u32, u32, u32, vp, sz, vp, u32, vp, sz, sz,
                                   ctypes.POINTER(i32), i32]
    lib.orc_interpolate.argtypes = [u32, u32, u32, vp, sz, vp, u32, vp, sz, sz, i32]
    return lib


def _pins_hold(lib) -> bool:
    n, k, W = 16, 6, 2
    rng = np.random.default_rng(13)
    src = rng.integers(0, 65536, (k, W), dtype=np.uint16)
    enc = np.empty((n, W), dtype=np.uint32)
    lib.orc_encode_sys(n, k, 0, src.ctypes.data, W, n, enc.ctypes.data, W, W, 1)
    for c in range(W):
        if list(enc[:, c]) != _gauss_codeword(src[:, c], n, k, n):
            return False
    pos = np.array([1, 4, 5, 9, 12, 15], dtype=np.uint32)
    v = rng.integers(0, P, (k, W), dtype=np.uint32)
    coef = np.empty((k, W), dtype=np.uint32)
    lib.orc_interpolate(n, k, 0, v.ctypes.data, W, pos.ctypes.data, k, coef.ctypes.data, W, W, 1)
    for c in range(W):
        if list(coef[:, c]) != small.gauss_decode([int(t) for t in v[:, c]],
                                                  [int(z) for z in pos], n, k):
            return False
    rec = np.ascontiguousarray(enc[pos])
    out = np.empty((k, W), dtype=np.uint16)
    flag = ctypes.c_int(0)
    lib.orc_decode_sys(n, k, 0, rec.ctypes.data, W, pos.ctypes.data, k, out.ctypes.data, W, W,
                       ctypes.byref(flag), 1)
    return bool(np.array_equal(out, src))


def test_unmutated_systematic_oracle_passes(tmp_path):
    path = tmp_path / "clean.c"
    path.write_text(open(SRC).read())
    assert _pins_hold(_lib(path, tmp_path / "clean.so"))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_systematic_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(text.replace(old, new))
    assert not _pins_hold(_lib(path, tmp_path / f"{name}.so"))
