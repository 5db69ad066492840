"""Planted mistakes: each plausible slip in the C oracle must fail a pin.

A mutant is a copy of ``oracle/fnt_rs_oracle.c`` with one textual change,
compiled into a temporary library on the CPU.  The checks below are the same
facts the pin tests use (DFT by definition, Gaussian elimination, MDS
recovery, root order), so a pass here shows those pins can see the slip.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import small

P = 65537
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "fnt_rs_oracle.c")

MUTANTS = {
    # transposed operand: coefficients taken in reverse order
    "horner_reversed": ("src[(size_t)i * ld_src + c]", "src[(size_t)(k - 1 - i) * ld_src + c]"),
    # wrong root: order 2n instead of n
    "root_order_2n": ("return orc_pow(3, 65536u / n);", "return orc_pow(3, 32768u / n);"),
    # dropped sign in the locator's constant term
    "locator_sign": ("A[0] = orc_sub(0, orc_mul(x[i], A[0]));", "A[0] = orc_mul(x[i], A[0]);"),
    # wrong index in synthetic division
    "synthdiv_index": ("Q[j - 1] = orc_add(A[j], orc_mul(xi, Q[j]));",
                       "Q[j - 1] = orc_add(A[j - 1], orc_mul(xi, Q[j]));"),
    # dropped n^-1 in the inverse DFT
    "idft_no_scale": ("out[(size_t)j * ld_out + c] = inverse ? orc_mul(acc, ninv) : acc;",
                      "out[(size_t)j * ld_out + c] = acc;"),
    # derivative without the factor j
    "derivative_no_j": ("orc_mul(j % ORC_P, A[j])", "A[j]"),
}


def _build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) >= 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(text.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(path), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    u32, sz, i32, vp = ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p
    lib.orc_encode.argtypes = [u32, u32, u32, vp, sz, vp, sz, sz, i32]
    lib.orc_decode.argtypes = [u32, u32, u32, vp, sz, vp, u32, vp, sz, sz,
                               ctypes.POINTER(i32), i32]
    lib.orc_dft.argtypes = [u32, u32, i32, vp, sz, vp, sz, sz, i32]
    lib.orc_root.argtypes = [u32]
    lib.orc_root.restype = u32
    return lib


def _pins_hold(lib) -> bool:
    """The pin facts, evaluated on a (possibly mutated) oracle library."""
    rng = np.random.default_rng(11)
    n, k, W = 16, 6, 3
    # root order
    r = lib.orc_root(n)
    if pow(r, n, P) != 1 or pow(r, n // 2, P) != P - 1:
        return False
    # encode == DFT of zero-padded source
    s = rng.integers(1, 65536, size=(k, W), dtype=np.uint16)
    e = np.empty((n, W), dtype=np.uint32)
    lib.orc_encode(n, k, 0, s.ctypes.data, W, e.ctypes.data, W, W, 1)
    for c in range(W):
        if list(e[:, c]) != small.dft_definition([int(v) for v in s[:, c]] + [0] * (n - k),
                                                 small.root(n)):
            return False
    # inverse DFT definition
    x = rng.integers(0, P, size=(n, 1), dtype=np.uint32)
    y = np.empty_like(x)
    lib.orc_dft(n, 0, 1, x.ctypes.data, 1, y.ctypes.data, 1, 1, 1)
    if list(y[:, 0]) != small.dft_definition([int(v) for v in x[:, 0]], small.root(n), True):
        return False
    # interpolation == Gaussian elimination on arbitrary received values
    pos = np.array([1, 4, 5, 9, 12, 15], dtype=np.uint32)
    v = rng.integers(0, P, size=(k, W), dtype=np.uint32)
    out = np.empty((k, W), dtype=np.uint16)
    flag = ctypes.c_int(0)
    lib.orc_decode(n, k, 0, v.ctypes.data, W, pos.ctypes.data, k, out.ctypes.data, W, W,
                   ctypes.byref(flag), 1)
    for c in range(W):
        want = small.gauss_decode([int(t) for t in v[:, c]], [int(z) for z in pos], n, k)
        if list(out[:, c]) != [0 if w == 65536 else w for w in want]:
            return False
    return True


def test_unmutated_oracle_passes(tmp_path):
    text = open(SRC).read()
    path = tmp_path / "clean.c"
    path.write_text(text)
    so = tmp_path / "clean.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(path), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    u32, sz, i32, vp = ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p
    lib.orc_encode.argtypes = [u32, u32, u32, vp, sz, vp, sz, sz, i32]
    lib.orc_decode.argtypes = [u32, u32, u32, vp, sz, vp, u32, vp, sz, sz,
                               ctypes.POINTER(i32), i32]
    lib.orc_dft.argtypes = [u32, u32, i32, vp, sz, vp, sz, sz, i32]
    lib.orc_root.argtypes = [u32]
    lib.orc_root.restype = u32
    assert _pins_hold(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    assert not _pins_hold(_build_mutant(tmp_path, name))
