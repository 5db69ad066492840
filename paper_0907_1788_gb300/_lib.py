"""ctypes loader for libfntrs.so (the C ABI of include/fnt_rs.h).

The library is built in-tree by :mod:`paper_0907_1788_gb300.build`.  There is
no fallback of any kind: if the shared library is missing or fails to load,
every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# FNTRS_LIB selects another in-tree build of the same library (the debug
# build with device index checks); by default the release build is loaded.
LIB_PATH = os.environ.get("FNTRS_LIB") or os.path.join(HERE, "_build", "libfntrs.so")

_lock = threading.Lock()
_lib = None


class FntRsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = f"fnt_rs error {code}"
        if _lib is not None:
            msg += f" ({_lib.fnt_rs_strerror(code).decode()})"
        if what:
            msg = f"{what}: {msg}"
        super().__init__(msg)


def load(build_if_missing: bool = False):
    """Load libfntrs.so; raise if it is not built (or build it when asked)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise RuntimeError(
                    f"libfntrs.so not found at {LIB_PATH}; run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first")
            from . import build as _b
            _b.build()
        lib = ctypes.CDLL(LIB_PATH)
        vp, sz, u32, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_int
        sig = {
            "fnt_rs_plan_create": (i32, [ctypes.POINTER(vp), u32, u32, u32, u32, vp]),
            "fnt_rs_plan_destroy": (None, [vp]),
            "fnt_rs_workspace_bytes": (sz, [vp, sz, i32]),
            "fnt_rs_encode": (i32, [vp, vp, sz, vp, sz, sz, vp, vp]),
            "fnt_rs_decode_prepare": (i32, [vp, vp, u32, vp]),
            "fnt_rs_decode": (i32, [vp, vp, sz, vp, u32, vp, sz, sz, vp, vp]),
            "fnt_rs_decode_slots": (i32, [vp, vp, sz, vp, u32, vp, sz, sz, vp, vp]),
            "fnt_rs_decode_full": (i32, [vp, vp, sz, vp, sz, sz, vp, vp]),
            "fnt_rs_fnt": (i32, [vp, vp, sz, vp, sz, sz, i32, vp, vp]),
            "fnt_rs_encode_host": (i32, [vp, vp, vp, sz, vp, vp]),
            "fnt_rs_encode_noalloc": (i32, [vp, vp, sz, vp, sz, sz, vp]),
            "fnt_rs_debug_bounds": (i32, []),
            "fnt_rs_decode_host": (i32, [vp, vp, vp, u32, vp, sz, vp, vp]),
            "fnt_rs_plan_set_length": (i32, [vp, u32]),
            "fnt_rs_encode_sys": (i32, [vp, vp, sz, vp, sz, sz, vp, vp]),
            "fnt_rs_decode_sys": (i32, [vp, vp, sz, vp, u32, vp, sz, sz, vp, vp]),
            "fnt_rs_wire_escape_cap": (sz, [vp, sz]),
            "fnt_rs_encode_wire": (i32, [vp, vp, sz, vp, sz, sz, vp, u32, vp, vp, vp]),
            "fnt_rs_decode_wire": (i32, [vp, vp, sz, vp, u32, vp, u32, vp, sz, sz, vp, vp]),
            "fnt_rs_encode_wire_host": (i32, [vp, vp, vp, sz, vp, u32, ctypes.POINTER(u32),
                                              vp, vp]),
            "fnt_rs_decode_wire_host": (i32, [vp, vp, vp, u32, vp, u32, vp, sz, vp, vp]),
            "fnt_rs_set_schedule": (i32, [vp, i32, i32]),
            "fnt_rs_get_schedule": (i32, [vp, i32]),
            "fnt_rs_autotune": (i32, [vp, sz, i32, vp, i32, vp]),
            "fnt_rs_status": (i32, [vp, vp]),
            "fnt_rs_server_create": (i32, [ctypes.POINTER(vp), sz, u32, i32]),
            "fnt_rs_server_preplan": (i32, [vp, u32, u32]),
            "fnt_rs_server_submit": (i32, [vp, vp, ctypes.POINTER(ctypes.c_uint64)]),
            "fnt_rs_server_poll": (i32, [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
            "fnt_rs_server_drain": (i32, [vp]),
            "fnt_rs_server_fetch": (i32, [vp, ctypes.c_uint64, vp, vp]),
            "fnt_rs_server_release": (i32, [vp, ctypes.c_uint64]),
            "fnt_rs_server_stats": (i32, [vp, ctypes.POINTER(ctypes.c_double), i32]),
            "fnt_rs_server_destroy": (None, [vp]),
            "fnt_rs_server_replay": (i32, [vp, vp, vp, u32, vp, vp]),
            "fnt_rs_baseline_replay": (i32, [vp, vp, u32, vp, vp, vp]),
            "fnt_rs_ragged_create": (i32, [ctypes.POINTER(vp), vp, u32, u32, vp]),
            "fnt_rs_ragged_run": (i32, [vp, vp]),
            "fnt_rs_ragged_run_plain": (i32, [vp, vp]),
            "fnt_rs_ragged_status": (i32, [vp, vp]),
            "fnt_rs_ragged_info": (i32, [vp, ctypes.POINTER(i32), i32]),
            "fnt_rs_ragged_destroy": (None, [vp]),
            "fnt_rs_strerror": (ctypes.c_char_p, [i32]),
            "fnt_rs_launch_count": (ctypes.c_uint64, []),
            "fnt_rs_plan_info": (i32, [vp, ctypes.POINTER(i32), i32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class Group(ctypes.Structure):
    """fnt_rs_group of include/fnt_rs.h."""

    _fields_ = [("n", ctypes.c_uint32), ("k", ctypes.c_uint32), ("W", ctypes.c_size_t),
                ("src", ctypes.c_void_p), ("ld_src", ctypes.c_size_t),
                ("enc", ctypes.c_void_p), ("ld_enc", ctypes.c_size_t),
                ("positions", ctypes.c_void_p), ("npos", ctypes.c_uint32),
                ("out", ctypes.c_void_p), ("ld_out", ctypes.c_size_t)]


class TuneResult(ctypes.Structure):
    """fnt_rs_tune_result of include/fnt_rs.h."""

    _fields_ = [("sched", ctypes.c_int), ("us", ctypes.c_float)]


class Request(ctypes.Structure):
    """fnt_rs_request of include/fnt_rs.h."""

    _fields_ = [("op", ctypes.c_int), ("n", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("W", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("positions", ctypes.c_void_p), ("npos", ctypes.c_uint32)]


def declared_symbols():
    """Names declared with `extern "C"` linkage in include/fnt_rs.h."""
    import re

    hdr = os.path.join(os.path.dirname(HERE), "include", "fnt_rs.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"\b(fnt_rs_[a-z_]+)\s*\(", text)))
