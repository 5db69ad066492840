"""ctypes wrapper around the C oracle (``fnt_rs_oracle.c``).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

Layouts follow the interleaved packet layout of Sec. II.B (data units hold
one 2-byte symbol of many codewords): a batch of W codewords is a row-major
``[rows][W]`` array whose column c is codeword c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

P = 65537
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fnt_rs_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile ``fnt_rs_oracle.c`` with gcc (OpenMP over codewords)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC,
                               "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32, sz, i32 = ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int
            vp = ctypes.c_void_p
            lib.orc_pow.argtypes = [u32, ctypes.c_uint64]
            lib.orc_pow.restype = u32
            lib.orc_inv.argtypes = [u32]
            lib.orc_inv.restype = u32
            lib.orc_root.argtypes = [u32]
            lib.orc_root.restype = u32
            lib.orc_dft.argtypes = [u32, u32, i32, vp, sz, vp, sz, sz, i32]
            lib.orc_dft.restype = i32
            lib.orc_encode.argtypes = [u32, u32, u32, vp, sz, vp, sz, sz, i32]
            lib.orc_encode.restype = i32
            lib.orc_encode_rows.argtypes = [u32, u32, u32, vp, sz, vp, u32, vp, sz, sz, i32]
            lib.orc_encode_rows.restype = i32
            lib.orc_pattern.argtypes = [u32, u32, u32, vp, u32, vp, vp, vp]
            lib.orc_pattern.restype = i32
            lib.orc_decode.argtypes = [u32, u32, u32, vp, sz, vp, u32, vp, sz, sz,
                                       ctypes.POINTER(i32), i32]
            lib.orc_decode.restype = i32
            lib.orc_interpolate.argtypes = [u32, u32, u32, vp, sz, vp, u32, vp, sz, sz, i32]
            lib.orc_interpolate.restype = i32
            lib.orc_encode_sys.argtypes = [u32, u32, u32, vp, sz, u32, vp, sz, sz, i32]
            lib.orc_encode_sys.restype = i32
            lib.orc_decode_sys.argtypes = [u32, u32, u32, vp, sz, vp, u32, vp, sz, sz,
                                           ctypes.POINTER(i32), i32]
            lib.orc_decode_sys.restype = i32
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def max_threads() -> int:
    return int(_load().orc_max_threads())


def root(n: int) -> int:
    """Root of order n used by the code: 3^(65536/n) (Sec. II.B)."""
    return int(_load().orc_root(n))


def encode(src: np.ndarray, n: int, root_: int = 0, threads: int = 0) -> np.ndarray:
    """e_j = s(r^j) for every column of ``src`` ([k][W] uint16) -> [n][W] uint32."""
    src = np.ascontiguousarray(src, dtype=np.uint16)
    k, W = src.shape
    out = np.empty((n, W), dtype=np.uint32)
    rc = _load().orc_encode(n, k, root_, _ptr(src), W, _ptr(out), W, W, threads or max_threads())
    if rc:
        raise ValueError(f"orc_encode failed: {rc}")
    return out


def encode_rows(src: np.ndarray, n: int, rows, root_: int = 0, threads: int = 0) -> np.ndarray:
    """e_j = s(r^j) at the given rows only: [len(rows)][W] uint32."""
    src = np.ascontiguousarray(src, dtype=np.uint16)
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    k, W = src.shape
    out = np.empty((len(rows), W), dtype=np.uint32)
    rc = _load().orc_encode_rows(n, k, root_, _ptr(src), W, _ptr(rows), len(rows), _ptr(out), W,
                                 W, threads or max_threads())
    if rc:
        raise ValueError(f"orc_encode_rows failed: {rc}")
    return out


def dft(x: np.ndarray, inverse: bool = False, root_: int = 0, threads: int = 0) -> np.ndarray:
    """DFT by definition of every column of ``x`` ([n][W] uint32)."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    n, W = x.shape
    out = np.empty((n, W), dtype=np.uint32)
    rc = _load().orc_dft(n, root_, int(inverse), _ptr(x), W, _ptr(out), W, W,
                         threads or max_threads())
    if rc:
        raise ValueError(f"orc_dft failed: {rc}")
    return out


def pattern(n: int, k: int, positions, root_: int = 0):
    """Return (A[0..k], A'(x_i), 1/A'(x_i)) for the first k positions."""
    pos = np.ascontiguousarray(positions, dtype=np.uint32)
    A = np.empty(k + 1, dtype=np.uint32)
    dA = np.empty(k, dtype=np.uint32)
    w = np.empty(k, dtype=np.uint32)
    rc = _load().orc_pattern(n, k, root_, _ptr(pos), len(pos), _ptr(A), _ptr(dA), _ptr(w))
    if rc:
        raise ValueError(f"orc_pattern failed: {rc}")
    return A, dA, w


def decode(recv: np.ndarray, positions, n: int, k: int, root_: int = 0, threads: int = 0):
    """Interpolate every column of ``recv`` ([npos][W] uint32).

    Returns (source [k][W] uint16, range_flag).  A coefficient equal to 65536
    is written as 0 and sets ``range_flag``.
    """
    recv = np.ascontiguousarray(recv, dtype=np.uint32)
    pos = np.ascontiguousarray(positions, dtype=np.uint32)
    npos, W = recv.shape
    if len(pos) != npos:
        raise ValueError("one received row per position")
    out = np.empty((k, W), dtype=np.uint16)
    flag = ctypes.c_int(0)
    rc = _load().orc_decode(n, k, root_, _ptr(recv), W, _ptr(pos), npos, _ptr(out), W, W,
                            ctypes.byref(flag), threads or max_threads())
    if rc not in (0, -3):
        raise ValueError(f"orc_decode failed: {rc}")
    return out, bool(flag.value)


def interpolate(recv: np.ndarray, positions, n: int, k: int, root_: int = 0,
                threads: int = 0) -> np.ndarray:
    """Coefficients of the interpolant of the first k received points: [k][W] uint32 in [0, p)."""
    recv = np.ascontiguousarray(recv, dtype=np.uint32)
    pos = np.ascontiguousarray(positions, dtype=np.uint32)
    npos, W = recv.shape
    if len(pos) != npos:
        raise ValueError("one received row per position")
    out = np.empty((k, W), dtype=np.uint32)
    rc = _load().orc_interpolate(n, k, root_, _ptr(recv), W, _ptr(pos), npos, _ptr(out), W, W,
                                 threads or max_threads())
    if rc:
        raise ValueError(f"orc_interpolate failed: {rc}")
    return out


def encode_sys(src: np.ndarray, n: int, n_out: int = 0, root_: int = 0,
               threads: int = 0) -> np.ndarray:
    """Systematic code: [n_out][W] uint32 whose first k rows are ``src`` ([k][W] uint16)."""
    src = np.ascontiguousarray(src, dtype=np.uint16)
    k, W = src.shape
    n_out = n_out or n
    out = np.empty((n_out, W), dtype=np.uint32)
    rc = _load().orc_encode_sys(n, k, root_, _ptr(src), W, n_out, _ptr(out), W, W,
                                threads or max_threads())
    if rc:
        raise ValueError(f"orc_encode_sys failed: {rc}")
    return out


def decode_sys(recv: np.ndarray, positions, n: int, k: int, root_: int = 0, threads: int = 0):
    """Systematic decode: (source [k][W] uint16, range_flag) from the first k received points."""
    recv = np.ascontiguousarray(recv, dtype=np.uint32)
    pos = np.ascontiguousarray(positions, dtype=np.uint32)
    npos, W = recv.shape
    if len(pos) != npos:
        raise ValueError("one received row per position")
    out = np.empty((k, W), dtype=np.uint16)
    flag = ctypes.c_int(0)
    rc = _load().orc_decode_sys(n, k, root_, _ptr(recv), W, _ptr(pos), npos, _ptr(out), W, W,
                                ctypes.byref(flag), threads or max_threads())
    if rc not in (0, -3):
        raise ValueError(f"orc_decode_sys failed: {rc}")
    return out, bool(flag.value)
