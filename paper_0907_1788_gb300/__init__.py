"""GB300-native FNT-based Reed-Solomon erasure codes over F_65537.

Python binding of ``libfntrs.so`` (C ABI in ``include/fnt_rs.h``).  The
functions below carry the C names and only marshal arguments: torch tensors
supply device memory and streams, every arithmetic step runs in the library's
CUDA kernels.  There is no CPU path.

Layout (Sec. II.B interleaving): a batch of W codewords is a row-major
``[rows][W]`` tensor whose column c is codeword c --
source ``[k][W]`` 16-bit, encoded ``[n][W]`` 32-bit (values 0..65536),
received ``[npos][W]`` 32-bit, decoded ``[k][W]`` 16-bit.  Any torch dtype of
the right width works (the library reads raw bits); the helpers allocate
int16 / int32 tensors, which torch supports fully, holding the unsigned values.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib import FntRsError, Group, LIB_PATH, Request, load  # noqa: F401

P = 65537
OP_ENCODE, OP_DECODE, OP_FNT, OP_ENCODE_HOST, OP_DECODE_HOST = 0, 1, 2, 3, 4
OP_ENCODE_SYS, OP_DECODE_SYS = 5, 6
OP_ENCODE_WIRE, OP_DECODE_WIRE, OP_ENCODE_WIRE_HOST, OP_DECODE_WIRE_HOST = 7, 8, 9, 10
SCHED_AUTO, SCHED_TMA, SCHED_TILE, SCHED_SPLIT, SCHED_CPA, SCHED_PAPER = 0, 1, 2, 3, 4, 5
SCHED_DIRECT = 6
SCHED_NAMES = {SCHED_TMA: "tma", SCHED_TILE: "tile", SCHED_SPLIT: "split", SCHED_CPA: "cpa",
               SCHED_PAPER: "paper", SCHED_DIRECT: "direct"}

E_RANGE = -7
E_TIMEOUT = -8
E_BOUNDS = -10


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _check(rc: int, what: str):
    if rc != 0:
        raise FntRsError(rc, what)


def _cols(t: torch.Tensor):
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a 2-D row-major tensor with unit column stride")
    return t.shape[1], t.stride(0)


def _positions(positions) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(positions, dtype=np.uint32))


def fnt_rs_plan_create(n: int, k: int, p: int = P, root: int = 0, stream=None) -> int:
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.fnt_rs_plan_create(ctypes.byref(h), n, k, p, root, _stream(stream)),
           "fnt_rs_plan_create")
    return h.value


def fnt_rs_plan_destroy(plan: int) -> None:
    load().fnt_rs_plan_destroy(plan)


def fnt_rs_workspace_bytes(plan: int, W: int, op: int) -> int:
    return int(load().fnt_rs_workspace_bytes(plan, W, op))


def fnt_rs_encode(plan, src: torch.Tensor, enc: torch.Tensor, workspace=None, stream=None):
    W, ld_src = _cols(src)
    W2, ld_enc = _cols(enc)
    if W2 != W:
        raise ValueError("src and enc must have the same number of columns")
    _check(load().fnt_rs_encode(plan, _ptr(src), ld_src, _ptr(enc), ld_enc, W, _ptr(workspace),
                                _stream(stream)), "fnt_rs_encode")


def fnt_rs_decode_prepare(plan, positions, stream=None):
    pos = _positions(positions)
    _check(load().fnt_rs_decode_prepare(plan, pos.ctypes.data, len(pos), _stream(stream)),
           "fnt_rs_decode_prepare")


def fnt_rs_decode(plan, recv: torch.Tensor, positions, out: torch.Tensor, workspace=None,
                  stream=None):
    W, ld_recv = _cols(recv)
    W2, ld_out = _cols(out)
    if W2 != W:
        raise ValueError("recv and out must have the same number of columns")
    pos = _positions(positions)
    _check(load().fnt_rs_decode(plan, _ptr(recv), ld_recv, pos.ctypes.data, len(pos), _ptr(out),
                                ld_out, W, _ptr(workspace), _stream(stream)), "fnt_rs_decode")


def fnt_rs_decode_slots(plan, slots: torch.Tensor, positions, out: torch.Tensor, workspace=None,
                        stream=None):
    W, ld = _cols(slots)
    W2, ld_out = _cols(out)
    if W2 != W:
        raise ValueError("slots and out must have the same number of columns")
    pos = _positions(positions)
    _check(load().fnt_rs_decode_slots(plan, _ptr(slots), ld, pos.ctypes.data, len(pos), _ptr(out),
                                      ld_out, W, _ptr(workspace), _stream(stream)),
           "fnt_rs_decode_slots")


def fnt_rs_decode_full(plan, enc: torch.Tensor, out: torch.Tensor, workspace=None, stream=None):
    W, ld = _cols(enc)
    W2, ld_out = _cols(out)
    if W2 != W:
        raise ValueError("enc and out must have the same number of columns")
    _check(load().fnt_rs_decode_full(plan, _ptr(enc), ld, _ptr(out), ld_out, W, _ptr(workspace),
                                     _stream(stream)), "fnt_rs_decode_full")


def fnt_rs_fnt(plan, x: torch.Tensor, out: torch.Tensor, inverse: bool = False, workspace=None,
               stream=None):
    W, ld_in = _cols(x)
    W2, ld_out = _cols(out)
    if W2 != W:
        raise ValueError("in and out must have the same number of columns")
    _check(load().fnt_rs_fnt(plan, _ptr(x), ld_in, _ptr(out), ld_out, W, int(bool(inverse)),
                             _ptr(workspace), _stream(stream)), "fnt_rs_fnt")


def fnt_rs_encode_host(plan, h_src: torch.Tensor, h_enc: torch.Tensor, workspace, stream=None):
    W = h_src.shape[1]
    _check(load().fnt_rs_encode_host(plan, _ptr(h_src), _ptr(h_enc), W, _ptr(workspace),
                                     _stream(stream)), "fnt_rs_encode_host")


def fnt_rs_decode_host(plan, h_recv: torch.Tensor, positions, h_out: torch.Tensor, workspace,
                       stream=None):
    W = h_recv.shape[1]
    pos = _positions(positions)
    _check(load().fnt_rs_decode_host(plan, _ptr(h_recv), pos.ctypes.data, len(pos), _ptr(h_out),
                                     W, _ptr(workspace), _stream(stream)), "fnt_rs_decode_host")


def fnt_rs_encode_noalloc(plan, src: torch.Tensor, enc: torch.Tensor, stream=None):
    """fnt_rs_encode without a workspace: scratch comes from the library's fixed device array.

    For callers that cannot allocate device memory while running (all memory
    reserved up front, or no cudaMalloc allowed on the hot path).  Requests
    whose encode workspace (fnt_rs_workspace_bytes: n * W * 4 for a long
    code, about twice that for a punctured one) is above
    FNT_RS_NOALLOC_SCRATCH_BYTES raise FntRsError (code -9) before anything
    is launched; concurrent calls on different streams share the scratch.
    """
    W, ld_src = _cols(src)
    W2, ld_enc = _cols(enc)
    if W2 != W:
        raise ValueError("src and enc must have the same number of columns")
    _check(load().fnt_rs_encode_noalloc(plan, _ptr(src), ld_src, _ptr(enc), ld_enc, W,
                                        _stream(stream)), "fnt_rs_encode_noalloc")


NOALLOC_SCRATCH_BYTES = 16 << 20


def fnt_rs_ragged_create(groups, nstreams: int = 8, stream=None) -> int:
    """groups: sequence of dicts with n, k, src, enc and optional positions, out (tensors)."""
    arr = (Group * len(groups))()
    keep = []
    for i, g in enumerate(groups):
        W, ld_src = _cols(g["src"])
        _, ld_enc = _cols(g["enc"])
        e = arr[i]
        e.n, e.k, e.W = g["n"], g["k"], W
        e.src, e.ld_src = _ptr(g["src"]), ld_src
        e.enc, e.ld_enc = _ptr(g["enc"]), ld_enc
        if g.get("positions") is not None:
            pos = _positions(g["positions"])
            keep.append(pos)
            e.positions, e.npos = pos.ctypes.data, len(pos)
            _, ld_out = _cols(g["out"])
            e.out, e.ld_out = _ptr(g["out"]), ld_out
    h = ctypes.c_void_p()
    _check(load().fnt_rs_ragged_create(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p),
                                       len(groups), nstreams, _stream(stream)),
           "fnt_rs_ragged_create")
    return h.value


def fnt_rs_ragged_run(r, stream=None):
    _check(load().fnt_rs_ragged_run(r, _stream(stream)), "fnt_rs_ragged_run")


def fnt_rs_ragged_run_plain(r, stream=None):
    _check(load().fnt_rs_ragged_run_plain(r, _stream(stream)), "fnt_rs_ragged_run_plain")


def fnt_rs_ragged_status(r, stream=None) -> int:
    return int(load().fnt_rs_ragged_status(r, _stream(stream)))


def fnt_rs_ragged_info(r) -> dict:
    buf = (ctypes.c_int * 6)()
    m = load().fnt_rs_ragged_info(r, buf, 6)
    return dict(zip(["groups", "plans", "streams", "persistent_groups", "persistent_items",
                     "tuned_plans"], [int(buf[i]) for i in range(m)]))


def fnt_rs_ragged_destroy(r):
    load().fnt_rs_ragged_destroy(r)


def _requests(reqs):
    """Marshal request dicts (op, n, k, W, seed, positions) into a ctypes array."""
    arr = (Request * len(reqs))()
    keep = []
    for i, q in enumerate(reqs):
        e = arr[i]
        e.op = OP_DECODE if q["op"] == "decode" else OP_ENCODE
        e.n, e.k, e.W, e.seed = q["n"], q["k"], q["W"], q["seed"]
        if q.get("positions") is not None:
            pos = _positions(q["positions"])
            keep.append(pos)
            e.positions, e.npos = pos.ctypes.data, len(pos)
    return arr, keep


def fnt_rs_server_create(budget_bytes: int, nstreams: int = 8, keep_results: bool = True) -> int:
    h = ctypes.c_void_p()
    _check(load().fnt_rs_server_create(ctypes.byref(h), budget_bytes, nstreams,
                                       int(keep_results)), "fnt_rs_server_create")
    return h.value


def fnt_rs_server_preplan(server, n: int, k: int):
    _check(load().fnt_rs_server_preplan(server, n, k), "fnt_rs_server_preplan")


def fnt_rs_server_submit(server, req: dict) -> int:
    arr, keep = _requests([req])
    t = ctypes.c_uint64()
    _check(load().fnt_rs_server_submit(server, ctypes.cast(arr, ctypes.c_void_p),
                                       ctypes.byref(t)), "fnt_rs_server_submit")
    return t.value


def fnt_rs_server_poll(server, ticket: int):
    lat = ctypes.c_double(0)
    rc = load().fnt_rs_server_poll(server, ticket, ctypes.byref(lat))
    if rc < 0:
        raise FntRsError(rc, "fnt_rs_server_poll")
    return (rc == 1), lat.value


def fnt_rs_server_drain(server):
    _check(load().fnt_rs_server_drain(server), "fnt_rs_server_drain")


def fnt_rs_server_fetch(server, ticket: int, req: dict):
    """Return (input, output) host arrays of a finished request."""
    n, k, W = req["n"], req["k"], req["W"]
    if req["op"] == "encode":
        h_in, h_out = np.empty((k, W), np.uint16), np.empty((n, W), np.uint32)
    else:
        h_in, h_out = np.empty((k, W), np.uint32), np.empty((k, W), np.uint16)
    _check(load().fnt_rs_server_fetch(server, ticket, h_in.ctypes.data, h_out.ctypes.data),
           "fnt_rs_server_fetch")
    return h_in, h_out


def fnt_rs_server_release(server, ticket: int):
    _check(load().fnt_rs_server_release(server, ticket), "fnt_rs_server_release")


def fnt_rs_server_stats(server) -> dict:
    buf = (ctypes.c_double * 5)()
    m = load().fnt_rs_server_stats(server, buf, 5)
    keys = ["completed", "rejected", "arena_used", "arena_bytes", "plans"]
    return {keys[i]: buf[i] for i in range(m)}


def fnt_rs_server_destroy(server):
    load().fnt_rs_server_destroy(server)


def fnt_rs_server_replay(server, reqs, arrivals):
    """Replay a timed trace; returns (latency_ms array, wall seconds)."""
    arr, keep = _requests(reqs)
    t = np.ascontiguousarray(arrivals, dtype=np.float64)
    lat = np.zeros(len(reqs), dtype=np.float64)
    wall = ctypes.c_double(0)
    _check(load().fnt_rs_server_replay(server, ctypes.cast(arr, ctypes.c_void_p), t.ctypes.data,
                                       len(reqs), lat.ctypes.data, ctypes.byref(wall)),
           "fnt_rs_server_replay")
    return lat, wall.value


def fnt_rs_baseline_replay(reqs, arrivals, stream=None):
    arr, keep = _requests(reqs)
    t = np.ascontiguousarray(arrivals, dtype=np.float64)
    lat = np.zeros(len(reqs), dtype=np.float64)
    wall = ctypes.c_double(0)
    _check(load().fnt_rs_baseline_replay(ctypes.cast(arr, ctypes.c_void_p), t.ctypes.data,
                                         len(reqs), lat.ctypes.data, ctypes.byref(wall),
                                         _stream(stream)), "fnt_rs_baseline_replay")
    return lat, wall.value


def fnt_rs_plan_set_length(plan, n_out: int) -> None:
    _check(load().fnt_rs_plan_set_length(plan, n_out), "fnt_rs_plan_set_length")


def fnt_rs_encode_sys(plan, src: torch.Tensor, enc: torch.Tensor, workspace=None, stream=None):
    W, ld_src = _cols(src)
    W2, ld_enc = _cols(enc)
    if W2 != W:
        raise ValueError("src and enc must have the same number of columns")
    _check(load().fnt_rs_encode_sys(plan, _ptr(src), ld_src, _ptr(enc), ld_enc, W,
                                    _ptr(workspace), _stream(stream)), "fnt_rs_encode_sys")


def fnt_rs_decode_sys(plan, recv: torch.Tensor, positions, out: torch.Tensor, workspace=None,
                      stream=None):
    W, ld_recv = _cols(recv)
    W2, ld_out = _cols(out)
    if W2 != W:
        raise ValueError("recv and out must have the same number of columns")
    pos = _positions(positions)
    _check(load().fnt_rs_decode_sys(plan, _ptr(recv), ld_recv, pos.ctypes.data, len(pos),
                                    _ptr(out), ld_out, W, _ptr(workspace), _stream(stream)),
           "fnt_rs_decode_sys")


def fnt_rs_wire_escape_cap(plan, W: int) -> int:
    return int(load().fnt_rs_wire_escape_cap(plan, W))


def fnt_rs_encode_wire(plan, src: torch.Tensor, enc: torch.Tensor, esc: torch.Tensor,
                       esc_count: torch.Tensor, workspace=None, stream=None):
    """16-bit wire encode: enc [n_out][W] 16-bit, esc [cap][2] 32-bit {row, col} pairs
    (unordered), esc_count one 32-bit device word (may exceed cap)."""
    W, ld_src = _cols(src)
    W2, ld_enc = _cols(enc)
    if W2 != W:
        raise ValueError("src and enc must have the same number of columns")
    if esc.dim() != 2 or esc.shape[1] != 2 or not esc.is_contiguous():
        raise ValueError("esc must be a contiguous [cap][2] tensor")
    _check(load().fnt_rs_encode_wire(plan, _ptr(src), ld_src, _ptr(enc), ld_enc, W, _ptr(esc),
                                     esc.shape[0], _ptr(esc_count), _ptr(workspace),
                                     _stream(stream)), "fnt_rs_encode_wire")


def fnt_rs_decode_wire(plan, recv: torch.Tensor, positions, esc: torch.Tensor, nesc: int,
                       out: torch.Tensor, workspace=None, stream=None):
    """16-bit wire decode: recv [npos][W] 16-bit, esc [>= nesc][2] device {row, col} pairs."""
    W, ld_recv = _cols(recv)
    W2, ld_out = _cols(out)
    if W2 != W:
        raise ValueError("recv and out must have the same number of columns")
    if esc is not None and (esc.dim() != 2 or esc.shape[1] != 2 or not esc.is_contiguous()
                            or esc.shape[0] < nesc):
        raise ValueError("esc must be a contiguous [>= nesc][2] tensor")
    pos = _positions(positions)
    _check(load().fnt_rs_decode_wire(plan, _ptr(recv), ld_recv, pos.ctypes.data, len(pos),
                                     _ptr(esc), nesc, _ptr(out), ld_out, W, _ptr(workspace),
                                     _stream(stream)), "fnt_rs_decode_wire")


def fnt_rs_encode_wire_host(plan, h_src: torch.Tensor, h_enc: torch.Tensor, h_esc: np.ndarray,
                            workspace, stream=None) -> int:
    """Host-buffer wire encode; returns the number of escapes written (sorted) to h_esc."""
    W = h_src.shape[1]
    if h_esc.dtype != np.uint32 or h_esc.ndim != 2 or h_esc.shape[1] != 2 or \
            not h_esc.flags.c_contiguous:
        raise ValueError("h_esc must be a C-contiguous uint32 [cap][2] array")
    cnt = ctypes.c_uint32(0)
    _check(load().fnt_rs_encode_wire_host(plan, _ptr(h_src), _ptr(h_enc), W, h_esc.ctypes.data,
                                          h_esc.shape[0], ctypes.byref(cnt), _ptr(workspace),
                                          _stream(stream)), "fnt_rs_encode_wire_host")
    return cnt.value


def fnt_rs_decode_wire_host(plan, h_recv: torch.Tensor, positions, h_esc: np.ndarray,
                            h_out: torch.Tensor, workspace, stream=None):
    W = h_recv.shape[1]
    pos = _positions(positions)
    h_esc = np.ascontiguousarray(np.asarray(h_esc, dtype=np.uint32).reshape(-1, 2))
    _check(load().fnt_rs_decode_wire_host(plan, _ptr(h_recv), pos.ctypes.data, len(pos),
                                          h_esc.ctypes.data, len(h_esc), _ptr(h_out), W,
                                          _ptr(workspace), _stream(stream)),
           "fnt_rs_decode_wire_host")


def fnt_rs_set_schedule(plan, op: int, sched: int) -> None:
    _check(load().fnt_rs_set_schedule(plan, op, sched), "fnt_rs_set_schedule")


def fnt_rs_get_schedule(plan, op: int) -> int:
    rc = int(load().fnt_rs_get_schedule(plan, op))
    if rc < 0:
        _check(rc, "fnt_rs_get_schedule")
    return rc


def fnt_rs_autotune(plan, W: int, op: int, stream=None) -> list:
    """Times every schedule of `op` for W codewords; returns [(sched, us)], keeps the fastest."""
    from ._lib import TuneResult

    buf = (TuneResult * 8)()
    rc = int(load().fnt_rs_autotune(plan, W, op, buf, 8, _stream(stream)))
    if rc < 0:
        _check(rc, "fnt_rs_autotune")
    return [(int(buf[i].sched), float(buf[i].us)) for i in range(rc)]


def fnt_rs_status(plan, stream=None) -> int:
    return int(load().fnt_rs_status(plan, _stream(stream)))


def fnt_rs_debug_bounds() -> int:
    """1 if the loaded library is the debug build with device index checks."""
    return int(load().fnt_rs_debug_bounds())


def fnt_rs_strerror(code: int) -> str:
    return load().fnt_rs_strerror(code).decode()


def fnt_rs_launch_count() -> int:
    return int(load().fnt_rs_launch_count())


def fnt_rs_plan_info(plan) -> dict:
    buf = (ctypes.c_int * 8)()
    m = load().fnt_rs_plan_info(plan, buf, 8)
    keys = ["n", "k", "L", "C", "wt_one", "wt_two", "blocked", "patterns"]
    return {keys[i]: int(buf[i]) for i in range(m)}


class Plan:
    """Owns a plan handle; allocates outputs and workspace with torch (plumbing only)."""

    def __init__(self, n: int, k: int, root: int = 0, device=None, stream=None):
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.handle = fnt_rs_plan_create(n, k, P, root, stream)
        self.n, self.k = n, k
        self._ws = {}

    def close(self):
        if getattr(self, "handle", None):
            fnt_rs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, W: int, op: int):
        nbytes = fnt_rs_workspace_bytes(self.handle, W, op)
        if nbytes == 0:
            return None
        ws = self._ws.get(op)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self._ws[op] = ws
        return ws

    def encode(self, src: torch.Tensor, out=None, stream=None):
        W = src.shape[1]
        if out is None:
            out = torch.empty((getattr(self, "n_out", self.n), W), dtype=torch.int32,
                              device=src.device)
        fnt_rs_encode(self.handle, src, out, self.workspace(W, OP_ENCODE), stream)
        return out

    def prepare(self, positions, stream=None):
        fnt_rs_decode_prepare(self.handle, positions, stream)

    def decode(self, recv: torch.Tensor, positions, out=None, stream=None):
        W = recv.shape[1]
        if out is None:
            out = torch.empty((self.k, W), dtype=torch.int16, device=recv.device)
        fnt_rs_decode(self.handle, recv, positions, out, self.workspace(W, OP_DECODE), stream)
        return out

    def decode_slots(self, slots: torch.Tensor, positions, out=None, stream=None):
        W = slots.shape[1]
        if out is None:
            out = torch.empty((self.k, W), dtype=torch.int16, device=slots.device)
        fnt_rs_decode_slots(self.handle, slots, positions, out, self.workspace(W, OP_DECODE),
                            stream)
        return out

    def decode_full(self, enc: torch.Tensor, out=None, stream=None):
        W = enc.shape[1]
        if out is None:
            out = torch.empty((self.k, W), dtype=torch.int16, device=enc.device)
        fnt_rs_decode_full(self.handle, enc, out, self.workspace(W, OP_FNT), stream)
        return out

    def fnt(self, x: torch.Tensor, inverse: bool = False, out=None, stream=None):
        W = x.shape[1]
        if out is None:
            out = torch.empty((self.n, W), dtype=torch.int32, device=x.device)
        fnt_rs_fnt(self.handle, x, out, inverse, self.workspace(W, OP_FNT), stream)
        return out

    def status(self, stream=None) -> int:
        return fnt_rs_status(self.handle, stream)

    def set_length(self, n_out: int) -> None:
        """Puncture the code to its first n_out positions (n_out = n: the full code)."""
        fnt_rs_plan_set_length(self.handle, n_out)
        self.n_out = n_out

    def encode_sys(self, src: torch.Tensor, out=None, stream=None):
        W = src.shape[1]
        if out is None:
            out = torch.empty((getattr(self, "n_out", self.n), W), dtype=torch.int32,
                              device=src.device)
        fnt_rs_encode_sys(self.handle, src, out, self.workspace(W, OP_ENCODE_SYS), stream)
        return out

    def decode_sys(self, recv: torch.Tensor, positions, out=None, stream=None):
        W = recv.shape[1]
        if out is None:
            out = torch.empty((self.k, W), dtype=torch.int16, device=recv.device)
        fnt_rs_decode_sys(self.handle, recv, positions, out, self.workspace(W, OP_DECODE_SYS),
                          stream)
        return out

    def encode_wire(self, src: torch.Tensor, cap: int = 0, stream=None):
        """(symbols [n_out][W] 16-bit, escapes [m][2] {row, col} sorted) on the device.

        Reads the escape count back (synchronising the stream); a count above
        the capacity re-runs the encode with room for all of them.
        """
        W = src.shape[1]
        rows = getattr(self, "n_out", self.n)
        enc = torch.empty((rows, W), dtype=torch.int16, device=src.device)
        cap = cap or fnt_rs_wire_escape_cap(self.handle, W)
        cnt = torch.zeros(1, dtype=torch.int32, device=src.device)
        while True:
            esc = torch.empty((cap, 2), dtype=torch.int32, device=src.device)
            fnt_rs_encode_wire(self.handle, src, enc, esc, cnt,
                               self.workspace(W, OP_ENCODE_WIRE), stream)
            m = int(cnt.item())
            if m <= cap:
                break
            cap = m
        e = esc[:m].to(torch.int64)
        order = torch.argsort(e[:, 0] * (1 << 32) + e[:, 1])
        return enc, esc[:m][order].contiguous()

    def decode_wire(self, recv: torch.Tensor, positions, esc: torch.Tensor, out=None,
                    stream=None):
        W = recv.shape[1]
        if out is None:
            out = torch.empty((self.k, W), dtype=torch.int16, device=recv.device)
        nesc = 0 if esc is None else esc.shape[0]
        fnt_rs_decode_wire(self.handle, recv, positions, esc, nesc, out,
                           self.workspace(W, OP_DECODE_WIRE), stream)
        return out

    def autotune(self, W: int, op: int, stream=None) -> list:
        return fnt_rs_autotune(self.handle, W, op, stream)

    def schedule(self, op: int) -> int:
        return fnt_rs_get_schedule(self.handle, op)

    def set_schedule(self, op: int, sched: int) -> None:
        fnt_rs_set_schedule(self.handle, op, sched)

    def info(self) -> dict:
        return fnt_rs_plan_info(self.handle)


def to_device(a: np.ndarray, device="cuda") -> torch.Tensor:
    """Upload a uint16 / uint32 numpy array as an int16 / int32 tensor (same bits)."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(device)


def to_host(t: torch.Tensor) -> np.ndarray:
    """Download an int16 / int32 tensor as uint16 / uint32 numpy (same bits)."""
    a = t.detach().cpu().numpy()
    if a.dtype == np.int16:
        return a.view(np.uint16)
    if a.dtype == np.int32:
        return a.view(np.uint32)
    return a
