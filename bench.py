"""Benchmark: FNT-RS encode + per-pattern plan + erasure decode on GB300.

One step = one batch of the k=4096, n=8192, 2048-codeword workload (4 KB
packets, uniform random 16-bit source, one fresh uniform erasure pattern of
n-k positions per batch): encode the batch, build the pattern's decode plan
(steps 1-3), decode every codeword from the k received packets (stacked in
arrival order, the packed layout of the C ABI).

value = source bytes (k * W * 2) round-tripped per second (encode + plan +
decode), summed over ranks.  The timed steps run back to back with no L2
flush over source, encoded and decoded buffers that rotate over more memory
than L2 holds, so each step pays for its own write-back; a flushed pass is
reported beside it.  `--impl reference` times the CPU oracle on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = synth.CONFIGS["k4096_n8192_w2048"]
METRIC = "RS encode/decode source GB/s on 1 GB300 (% HBM roof, bit-exact); serving p50/p99 ms"
UNIT = "GB/s"
N_PATTERNS = 8  # more than the plan's 4 cached patterns: every step rebuilds
N_SETS = 3  # source / encoded / decoded buffer sets the timed steps rotate over


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


ISSUE_PEAK_TOPS = 152 * 4 * 32 * 2.07e9 / 1e12  # int32 lane-instructions / s (issue bound)


def fnt_instr(n: int) -> float:
    """Instructions of one length-n FNT in the minimal Z/(2^32-1) formulation.

    Radix-2 butterflies (n/2 log2 n) at 4 (add and sub, each with its carry
    fold), the power-of-two rotations of the radix <= 32 passes at 1, the
    general twiddles between passes at 3 (64-bit product + fold).
    """
    import math

    lg = int(math.log2(n))
    bfly = n // 2 * lg
    radices = {4096: [16, 16, 16], 8192: [32, 16, 16]}.get(n, [n])
    rot_per = {16: 17, 32: 49, 8: 5, 4: 1, 2: 0}
    rot = sum(n // r * rot_per.get(r, 0) for r in radices)
    tw = n * (len(radices) - 1)
    return 4 * bfly + rot + 3 * tw


def decode_instr(n: int, k: int) -> float:
    """Per codeword: three FNT_n + weights (k), A^ product (n), output reduction (k)."""
    return 3 * fnt_instr(n) + 3 * k + 3 * n + 4 * k


def encode_instr(n: int, k: int) -> float:
    """Per codeword: two FNT_(n/2) (k = n/2 classes) + class-1 twiddles + output reduction."""
    return 2 * fnt_instr(n // 2) + 3 * (n // 2) + 4 * n


# Sources that make up the device code of the workload's kernels (k_encode_tma,
# k_plan_fused, k_decode_tma at n = 8192): the kernel templates, the headers they
# include and the translation unit that instantiates them.
KERNEL_SOURCES = ("field.cuh", "tile.cuh", "kernels.cuh", "kargs.h", "logplan.cuh", "tma.cuh",
                  "sched.h", "inst.cuh", "inst_big.cu", "dbg.cuh")


def _src_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_0907_1788_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel sources still match."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        e = d.get(kernel)
        if e and e.get("src_hash") == _src_hash():
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


class Clocks:
    """Samples nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        import tempfile

        self.path = os.path.join(tempfile.gettempdir(),
                                 f"fntrs_clocks_rank{index}_{os.getpid()}.csv")

    def _lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            t0 = time.time()  # start timing only once sampling runs
            while self._lines() < 1 and time.time() - t0 < 5 and self.proc.poll() is None:
                time.sleep(0.02)
            self.start_line = self._lines()
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            n0 = self._lines()
            t0 = time.time()
            while self._lines() <= n0 and time.time() - t0 < 2 and self.proc.poll() is None:
                time.sleep(0.02)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = open(self.path).read().splitlines()
        for line in lines[max(0, getattr(self, "start_line", 1) - 1):]:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(seconds_target: float = 10.0):
    """The oracle as it stands on this host's cores, on a bounded sample."""
    import oracle

    cfg = WORKLOAD
    threads = oracle.max_threads()
    src = cfg.source()
    pos = cfg.positions()
    # pattern (steps 1-3 inside the oracle decode) costs O(k^2) once per batch
    t0 = time.perf_counter()
    oracle.pattern(cfg.n, cfg.k, pos)
    t_pat = time.perf_counter() - t0
    cols = max(threads, 1)
    sub = np.ascontiguousarray(src[:, :cols])
    t0 = time.perf_counter()
    enc = oracle.encode(sub, cfg.n, threads=threads)
    t_enc = time.perf_counter() - t0
    recv = np.ascontiguousarray(enc[pos])
    t0 = time.perf_counter()
    out, _ = oracle.decode(recv, pos, cfg.n, cfg.k, threads=threads)
    t_dec = time.perf_counter() - t0  # includes one pattern build
    assert np.array_equal(out, sub)
    per_cw = (t_enc + max(t_dec - t_pat, 0.0)) / cols
    per_batch = per_cw * cfg.W + t_pat
    gbs = cfg.k * cfg.W * 2 / per_batch / 1e9
    return {"value": gbs, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"{cols} codewords of {cfg.name} encoded (Horner) and decoded (Lagrange) on "
                       f"{threads} threads + one pattern build; scaled to the {cfg.W}-codeword "
                       f"batch: {per_batch:.2f} s per batch")}


def ragged_measure(pkg, dev, wave_bytes=32 << 30, nstreams=16, max_groups=None):
    """The whole seed-4 ragged batch (4096 groups) in memory-capped waves.

    Groups are taken in batch order into waves of at most `wave_bytes` of
    source, encoded and decoded buffers; each wave is one graph (one launch of
    the persistent kernel holding every group) timed against the same groups'
    per-group plain calls.  Times and bytes are summed over the waves."""
    import torch

    specs = synth.ragged_groups(seed=4, groups=4096)
    if max_groups:
        specs = specs[:max_groups]
    gen = torch.Generator(device=dev)
    gen.manual_seed(4)
    waves, cur, cur_bytes = [], [], 0
    for g in specs:
        size = g["k"] * g["W"] * 2 + g["n"] * g["W"] * 4 + g["k"] * g["W"] * 2
        if cur and cur_bytes + size > wave_bytes:
            waves.append(cur)
            cur, cur_bytes = [], 0
        cur.append(g)
        cur_bytes += size
    if cur:
        waves.append(cur)
    st = torch.cuda.current_stream()
    tot = {"groups": 0, "persistent_groups": 0, "items": 0, "graph_ms": 0.0, "plain_ms": 0.0,
           "source_bytes": 0, "buffer_bytes": 0}
    ok = True
    for wave in waves:
        groups = []
        for g in wave:
            n, k, W = g["n"], g["k"], g["W"]
            src = torch.randint(0, 65536, (k, W), generator=gen, device=dev, dtype=torch.int32)
            groups.append({"n": n, "k": k, "src": src.to(torch.int16),
                           "enc": torch.empty((n, W), dtype=torch.int32, device=dev),
                           "out": torch.empty((k, W), dtype=torch.int16, device=dev),
                           "positions": g["positions"]})
            tot["source_bytes"] += k * W * 2
            tot["buffer_bytes"] += k * W * 2 + n * W * 4 + k * W * 2
        r = pkg.fnt_rs_ragged_create(groups, nstreams=nstreams)
        try:
            def timed(fn, reps):
                ts = []
                for _ in range(reps):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(st)
                    fn(r, st)
                    b.record(st)
                    torch.cuda.synchronize()
                    ts.append(a.elapsed_time(b))
                return min(ts)

            tot["graph_ms"] += timed(pkg.fnt_rs_ragged_run, 2)
            tot["plain_ms"] += timed(pkg.fnt_rs_ragged_run_plain, 1)
            ok = ok and all(torch.equal(g["out"], g["src"])
                            for g in groups[:: max(1, len(groups) // 16)])
            ok = ok and pkg.fnt_rs_ragged_status(r) == 0
            info = pkg.fnt_rs_ragged_info(r)
            tot["groups"] += info["groups"]
            tot["persistent_groups"] += info["persistent_groups"]
            tot["items"] += info["persistent_items"]
        finally:
            pkg.fnt_rs_ragged_destroy(r)
        del groups
    src_bytes = tot["source_bytes"]
    return {"groups": tot["groups"], "persistent_groups": tot["persistent_groups"],
            "waves": len(waves), "wave_cap_gb": wave_bytes / 2**30,
            "persistent_items": tot["items"],
            "source_gb": src_bytes / 1e9, "buffers_gb": tot["buffer_bytes"] / 1e9,
            "graph_ms": tot["graph_ms"], "plain_ms": tot["plain_ms"],
            "graph_gbs": src_bytes / (tot["graph_ms"] * 1e-3) / 1e9,
            "plain_gbs": src_bytes / (tot["plain_ms"] * 1e-3) / 1e9,
            "round_trip_ok": bool(ok),
            "config": ("seed-4 ragged batch (n = 2^U{8..16}, k = floor(n*rho), rho in "
                       "{1/2,2/3,3/4,7/8}, W = 2^U{8..12}/2, own uniform pattern), all groups "
                       "in waves of at most the cap; each wave = one graph holding one launch of "
                       "the persistent kernel; each group = encode + pattern build + decode; "
                       "times summed over waves (min of 2 graph runs, 1 plain run per wave)")}


def serving_measure(pkg, rate=5000.0, count=3000, budget=32 << 30, patterns_per_shape=64):
    """Head of the seeded serving trace (Poisson arrivals at `rate` per second, encode
    and decode requests with n = 512..65536 at rates 1/2 and 3/4): continuous batching
    server vs one request at a time.

    Both arms count each request's latency from its scheduled arrival
    (replay start + arrival time) to the moment its result is seen, so
    queueing and any late submission are included on the same clock."""
    reqs = synth.serving_requests(seed=5, rate_per_s=rate, duration_s=count / rate * 2,
                                  patterns_per_shape=patterns_per_shape)[:count]
    trace = []
    for q in reqs:
        d = dict(op=q["op"], n=q["n"], k=q["k"], W=q["W"], seed=q["seed"])
        if q["op"] == "decode":
            d["positions"] = synth.received_positions(
                q["n"], synth.erased_uniform(q["pattern_seed"], q["n"], q["k"]))
        trace.append(d)
    arrivals = [q["t"] for q in reqs]
    src = sum(q["k"] * q["W"] * 2 for q in trace)
    srv = pkg.fnt_rs_server_create(budget, nstreams=16, keep_results=False)
    try:
        for n in sorted({q["n"] for q in trace}):
            for k in sorted({q["k"] for q in trace if q["n"] == n}):
                pkg.fnt_rs_server_preplan(srv, n, k)
        lat, wall = pkg.fnt_rs_server_replay(srv, trace, arrivals)
        stats = pkg.fnt_rs_server_stats(srv)
    finally:
        pkg.fnt_rs_server_destroy(srv)
    blat, bwall = pkg.fnt_rs_baseline_replay(trace, arrivals)
    ok = lat[lat >= 0]
    return {"rate_per_s": rate, "requests": len(trace), "completed": int(stats["completed"]),
            "rejected": int((lat < 0).sum()),
            "p50_ms": float(np.percentile(ok, 50)), "p99_ms": float(np.percentile(ok, 99)),
            "achieved_gbs": src / wall / 1e9, "wall_s": wall,
            "baseline": {"p50_ms": float(np.percentile(blat, 50)),
                         "p99_ms": float(np.percentile(blat, 99)),
                         "achieved_gbs": src / bwall / 1e9, "wall_s": bwall,
                         "kind": "one request at a time, plan + pattern built per request"},
            "budget_gb": budget / 2**30, "streams": 16,
            "latency_clock": "scheduled arrival -> result seen, both arms",
            "config": ("seed-5 Poisson trace (n = 2^U{9..16}, rho in {1/2,3/4}, packets "
                       f"2^U{{10..14}} B, half decode with {patterns_per_shape} recurring patterns "
                       f"per shape), first {len(trace)} requests; inputs generated on the device")}


def systematic_measure(pkg, dev, reps=20):
    """Systematic code on the headline shape: encode, decode with erasures, decode with
    every source position received (the direct path)."""
    import torch

    cfg = WORKLOAD
    n, k, W = cfg.n, cfg.k, cfg.W
    plan = pkg.Plan(n, k, device=dev)
    src = pkg.to_device(cfg.source(), dev)
    enc = plan.encode_sys(src)
    pos = cfg.positions()
    recv = torch.index_select(enc, 0, torch.from_numpy(pos.astype(np.int64)).to(dev))
    direct = np.arange(k, dtype=np.uint32)
    recv_d = enc[:k].contiguous()
    out = torch.empty((k, W), dtype=torch.int16, device=dev)
    ws_e = plan.workspace(W, pkg.OP_ENCODE_SYS)
    ws_d = plan.workspace(W, pkg.OP_DECODE_SYS)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for i in range(reps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    t_e = timed(lambda: pkg.fnt_rs_encode_sys(plan.handle, src, enc, ws_e))
    t_d = timed(lambda: pkg.fnt_rs_decode_sys(plan.handle, recv, pos, out, ws_d))
    ok = np.array_equal(pkg.to_host(out), cfg.source())
    t_dd = timed(lambda: pkg.fnt_rs_decode_sys(plan.handle, recv_d, direct, out, ws_d))
    ok = ok and np.array_equal(pkg.to_host(out), cfg.source()) and plan.status() == 0
    gb = k * W * 2 / 1e9
    return {"encode_sys_ms": t_e, "decode_sys_ms": t_d, "decode_sys_direct_ms": t_dd,
            "encode_sys_gbs": gb / (t_e * 1e-3), "decode_sys_gbs": gb / (t_d * 1e-3),
            "decode_sys_direct_gbs": gb / (t_dd * 1e-3), "round_trip_ok": bool(ok),
            "config": f"{cfg.name}, systematic code; decode with the step's erasure pattern "
                      "(pattern cached) and with positions 0..k-1 received; L2 flushed"}


def rate_measure(pkg, dev, n=8192, W=2048, reps=10):
    """Encode and decode at n = 8192 for the code rates of the ragged and serving
    workloads (k/n = 1/2, 2/3, 3/4, 7/8), pattern cached, L2 flushed."""
    import torch

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn):
        fn()
        ts = []
        for i in range(reps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    res = {}
    for num, den in ((1, 2), (2, 3), (3, 4), (7, 8)):
        k = n * num // den
        plan = pkg.Plan(n, k, device=dev)
        src = synth.source(k, k, W)
        d_src = pkg.to_device(src, dev)
        enc = torch.empty((n, W), dtype=torch.int32, device=dev)
        out = torch.empty((k, W), dtype=torch.int16, device=dev)
        ws_e = plan.workspace(W, pkg.OP_ENCODE)
        ws_d = plan.workspace(W, pkg.OP_DECODE)
        pos = synth.received_positions(n, synth.erased_uniform(k + 1, n, k))
        pkg.fnt_rs_encode(plan.handle, d_src, enc, ws_e)
        recv = torch.index_select(enc, 0, torch.from_numpy(pos.astype(np.int64)).to(dev))
        plan.prepare(pos)
        te = timed(lambda: pkg.fnt_rs_encode(plan.handle, d_src, enc, ws_e))
        td = timed(lambda: pkg.fnt_rs_decode(plan.handle, recv, pos, out, ws_d))
        ok = np.array_equal(pkg.to_host(out), src) and plan.status() == 0
        gb = k * W * 2 / 1e9
        res[f"{num}/{den}"] = {
            "k": k, "encode_ms": te, "decode_ms": td, "encode_gbs": gb / (te * 1e-3),
            "decode_gbs": gb / (td * 1e-3), "round_trip_ok": bool(ok),
            "schedules": {"encode": pkg.SCHED_NAMES[plan.schedule(pkg.OP_ENCODE)],
                          "decode": pkg.SCHED_NAMES[plan.schedule(pkg.OP_DECODE)]}}
        plan.close()
    res["config"] = f"n={n}, W={W}, uniform erasures, pattern cached, L2 flushed"
    return res


def large_code_measure(pkg, dev, reps=5):
    """The maximum length k = 32768, n = 65536 with 1024 codewords (2 KB packets), burst and
    uniform erasures: encode, pattern build and decode times (the split transforms)."""
    import torch

    res = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for name in ("k32768_n65536_w1024_burst", "k32768_n65536_w1024_uniform"):
        cfg = synth.CONFIGS[name]
        n, k, W = cfg.n, cfg.k, cfg.W
        plan = pkg.Plan(n, k, device=dev)
        src = cfg.source()
        d_src = pkg.to_device(src, dev)
        enc = torch.empty((n, W), dtype=torch.int32, device=dev)
        out = torch.empty((k, W), dtype=torch.int16, device=dev)
        ws_e = plan.workspace(W, pkg.OP_ENCODE)
        ws_d = plan.workspace(W, pkg.OP_DECODE)
        pos = cfg.positions()
        pkg.fnt_rs_encode(plan.handle, d_src, enc, ws_e)
        recv = torch.index_select(enc, 0, torch.from_numpy(pos.astype(np.int64)).to(dev))
        rng = np.random.default_rng(cfg.seed)

        def timed(fn):
            fn()
            ts = []
            for i in range(reps):
                flush.fill_(i & 0xFF)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            return statistics.median(ts)

        te = timed(lambda: pkg.fnt_rs_encode(plan.handle, d_src, enc, ws_e))
        # a fresh pattern each time (8 > 4 cached): the first k positions of new
        # permutations, drawn before the timed calls
        pats = iter([rng.permutation(n)[:k].astype(np.uint32) for _ in range(reps + 1)])
        tp = timed(lambda: plan.prepare(next(pats)))
        plan.prepare(pos)
        td = timed(lambda: pkg.fnt_rs_decode(plan.handle, recv, pos, out, ws_d))
        ok = np.array_equal(pkg.to_host(out), src) and plan.status() == 0
        gb = k * W * 2 / 1e9
        res[name] = {"encode_ms": te, "plan_ms": tp, "decode_ms": td,
                     "encode_gbs": gb / (te * 1e-3), "decode_gbs": gb / (td * 1e-3),
                     "decode_incl_plan_gbs": gb / ((td + tp) * 1e-3), "round_trip_ok": bool(ok),
                     "schedules": {"encode": pkg.SCHED_NAMES[plan.schedule(pkg.OP_ENCODE)],
                                   "decode": pkg.SCHED_NAMES[plan.schedule(pkg.OP_DECODE)]}}
        plan.close()
    res["config"] = ("L2 flushed between calls; the plan time is one fresh pattern's build, "
                     "host-side validation and upload included")
    return res


def direct_measure(pkg, dev, n=512, k=256, W=2048, reps=20):
    """The systematic code on a short code (k = 256, n = 512, 4 KB packets): the FNT
    route against the paper's direct (quadratic) encoder and decoder."""
    import torch

    src = synth.source(11, k, W)
    pos = synth.received_positions(n, synth.erased_uniform(12, n, k))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    res = {}
    for name, sched in (("fnt", pkg.SCHED_AUTO), ("direct", pkg.SCHED_DIRECT),
                        ("direct_simt", pkg.SCHED_DIRECT)):
        # the direct methods multiply on the tensor cores unless FNTRS_DIRECT_SIMT=1
        os.environ["FNTRS_DIRECT_SIMT"] = "1" if name == "direct_simt" else "0"
        plan = pkg.Plan(n, k, device=dev)
        plan.set_schedule(pkg.OP_ENCODE_SYS, sched)
        plan.set_schedule(pkg.OP_DECODE_SYS, sched)
        d_src = pkg.to_device(src, dev)
        enc = torch.empty((n, W), dtype=torch.int32, device=dev)
        out = torch.empty((k, W), dtype=torch.int16, device=dev)
        ws_e = plan.workspace(W, pkg.OP_ENCODE_SYS)
        ws_d = plan.workspace(W, pkg.OP_DECODE_SYS)
        pkg.fnt_rs_encode_sys(plan.handle, d_src, enc, ws_e)
        recv = torch.index_select(enc, 0, torch.from_numpy(pos.astype(np.int64)).to(dev))

        def timed(fn):
            for _ in range(3):
                fn()
            ts = []
            for i in range(reps):
                flush.fill_(i & 0xFF)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            return statistics.median(ts)

        te = timed(lambda: pkg.fnt_rs_encode_sys(plan.handle, d_src, enc, ws_e))
        td = timed(lambda: pkg.fnt_rs_decode_sys(plan.handle, recv, pos, out, ws_d))
        ok = np.array_equal(pkg.to_host(out), src) and plan.status() == 0
        gb = k * W * 2 / 1e9
        res[name] = {"encode_sys_ms": te, "decode_sys_ms": td, "encode_gbs": gb / (te * 1e-3),
                     "decode_gbs": gb / (td * 1e-3), "round_trip_ok": bool(ok)}
        plan.close()
    os.environ.pop("FNTRS_DIRECT_SIMT", None)
    res["products"] = {"direct": "tcgen05 BF16 limbs, FP32 accumulation in tensor memory",
                       "direct_simt": "integer kernel (64-bit accumulation)"}
    # the non-systematic code: FNT encode / 3-transform decode against the direct products
    code = {}
    for name, sched in (("fnt", pkg.SCHED_AUTO), ("direct", pkg.SCHED_DIRECT)):
        plan = pkg.Plan(n, k, device=dev)
        plan.set_schedule(pkg.OP_ENCODE, sched)
        plan.set_schedule(pkg.OP_DECODE, sched)
        d_src = pkg.to_device(src, dev)
        enc = torch.empty((n, W), dtype=torch.int32, device=dev)
        out = torch.empty((k, W), dtype=torch.int16, device=dev)
        ws_e = plan.workspace(W, pkg.OP_ENCODE)
        ws_d = plan.workspace(W, pkg.OP_DECODE)
        pkg.fnt_rs_encode(plan.handle, d_src, enc, ws_e)
        recv = torch.index_select(enc, 0, torch.from_numpy(pos.astype(np.int64)).to(dev))
        te = timed(lambda: pkg.fnt_rs_encode(plan.handle, d_src, enc, ws_e))
        td = timed(lambda: pkg.fnt_rs_decode(plan.handle, recv, pos, out, ws_d))
        ok = np.array_equal(pkg.to_host(out), src) and plan.status() == 0
        gb = k * W * 2 / 1e9
        code[name] = {"encode_ms": te, "decode_ms": td, "encode_gbs": gb / (te * 1e-3),
                      "decode_gbs": gb / (td * 1e-3), "round_trip_ok": bool(ok)}
        plan.close()
    res["nonsystematic"] = code
    res["config"] = (f"k={k}, n={n}, W={W} (4 KB packets), systematic code, uniform erasures "
                     "(pattern cached), L2 flushed")
    return res


def wire_measure(pkg, dev, reps=20):
    """16-bit wire format on the headline shape: device encode to 16-bit symbols +
    escapes, and decode from them (pattern cached), against the 32-bit calls."""
    import torch

    cfg = WORKLOAD
    n, k, W = cfg.n, cfg.k, cfg.W
    plan = pkg.Plan(n, k, device=dev)
    src = pkg.to_device(cfg.source(), dev)
    enc16 = torch.empty((n, W), dtype=torch.int16, device=dev)
    enc32 = torch.empty((n, W), dtype=torch.int32, device=dev)
    cap = pkg.fnt_rs_wire_escape_cap(plan.handle, W)
    esc = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    ws_e = plan.workspace(W, pkg.OP_ENCODE_WIRE)
    ws_e32 = plan.workspace(W, pkg.OP_ENCODE)
    pkg.fnt_rs_encode_wire(plan.handle, src, enc16, esc, cnt, ws_e)
    m = int(cnt.item())
    pos = cfg.positions()
    rank_of = torch.full((n,), -1, dtype=torch.int64, device=dev)
    pos_d = torch.from_numpy(pos.astype(np.int64)).to(dev)
    rank_of[pos_d] = torch.arange(len(pos), device=dev)
    e = esc[:m].to(torch.int64)
    keep = rank_of[e[:, 0]] >= 0
    r_esc = torch.stack([rank_of[e[keep, 0]], e[keep, 1]], 1).to(torch.int32).contiguous()
    recv16 = torch.index_select(enc16, 0, pos_d)
    out = torch.empty((k, W), dtype=torch.int16, device=dev)
    ws_d = plan.workspace(W, pkg.OP_DECODE_WIRE)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for i in range(reps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    t_e = timed(lambda: pkg.fnt_rs_encode_wire(plan.handle, src, enc16, esc, cnt, ws_e))
    t_e32 = timed(lambda: pkg.fnt_rs_encode(plan.handle, src, enc32, ws_e32))
    t_d = timed(lambda: pkg.fnt_rs_decode_wire(plan.handle, recv16, pos, r_esc, len(r_esc), out,
                                               ws_d))
    ok = np.array_equal(pkg.to_host(out), cfg.source()) and plan.status() == 0
    gb = k * W * 2 / 1e9
    return {"encode_wire_ms": t_e, "encode_u32_ms": t_e32, "decode_wire_ms": t_d,
            "encode_wire_gbs": gb / (t_e * 1e-3), "decode_wire_gbs": gb / (t_d * 1e-3),
            "escapes": m, "escapes_in_received_rows": int(len(r_esc)), "round_trip_ok": bool(ok),
            "config": f"{cfg.name}; 16-bit symbols + escape list; decode with the step's "
                      "erasure pattern (cached); L2 flushed"}


def paper_route_measure(pkg, dev, reps=10):
    """The paper's own decode route (chirp / middle products at length 2n, 4 FNT_2n per
    codeword) against the default decode (3 FNT_n) on the headline shape."""
    import torch

    cfg = WORKLOAD
    n, k, W = cfg.n, cfg.k, cfg.W
    pos = cfg.positions()
    src = cfg.source()
    out = torch.empty((k, W), dtype=torch.int16, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    res = {}
    for name, sched in (("default", None), ("paper", pkg.SCHED_PAPER)):
        plan = pkg.Plan(n, k, device=dev)
        if sched is not None:
            plan.set_schedule(pkg.OP_DECODE, sched)
        enc = plan.encode(pkg.to_device(src, dev))
        recv = torch.index_select(enc, 0, torch.from_numpy(pos.astype(np.int64)).to(dev))
        ws = plan.workspace(W, pkg.OP_DECODE)
        plan.prepare(pos)
        for _ in range(3):
            pkg.fnt_rs_decode(plan.handle, recv, pos, out, ws)
        ts = []
        for i in range(reps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            pkg.fnt_rs_decode(plan.handle, recv, pos, out, ws)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ok = np.array_equal(pkg.to_host(out), src) and plan.status() == 0
        res[name] = {"decode_ms": statistics.median(ts), "round_trip_ok": bool(ok),
                     "workspace_mb": (0 if ws is None else ws.numel()) / 1e6}
        plan.close()
    res["paper_over_default"] = res["paper"]["decode_ms"] / res["default"]["decode_ms"]
    res["transforms_per_codeword"] = {"default": "3 FNT_n", "paper": "4 FNT_2n (~8 FNT_n)"}
    res["config"] = f"{cfg.name}, pattern cached, L2 flushed"
    return res


def serving_sweep(pkg, rates=(5000.0, 10000.0, 20000.0, 50000.0), count=3000):
    """The serving trace at 5 k to 50 k requests per second, each on the head of its seeded trace, plus a
    fresh-pattern variant (every decode request brings a new erasure pattern)."""
    runs = [serving_measure(pkg, rate=r, count=count) for r in rates]
    fresh = serving_measure(pkg, rate=rates[0], count=count, patterns_per_shape=1 << 30)
    keep = ("rate_per_s", "requests", "rejected", "p50_ms", "p99_ms", "achieved_gbs")
    out = dict(runs[0])
    out["sweep"] = [dict({k: r[k] for k in keep},
                         baseline={k: r["baseline"][k] for k in ("p50_ms", "p99_ms", "achieved_gbs")})
                    for r in runs]
    out["fresh_patterns"] = dict({k: fresh[k] for k in keep},
                                 baseline={k: fresh["baseline"][k]
                                           for k in ("p50_ms", "p99_ms", "achieved_gbs")})
    return out


def max_over_ranks(x: float, device) -> float:
    """The slowest rank's value (a timing), or x itself without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(src_bytes_per_rank: int, world: int, ms: float) -> float:
    """Source GB/s of the whole job: every rank (a replica) decodes its own batch."""
    return world * src_bytes_per_rank / (ms * 1e-3) / 1e9


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    cfg = WORKLOAD
    threads = oracle.max_threads()
    src = cfg.source()
    pos = cfg.positions()
    cols = max(threads, 1)
    sub = np.ascontiguousarray(src[:, :cols])
    for _ in range(args.warmup):
        pass  # the oracle has no warm state; warm-up steps are not repeated
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        enc = oracle.encode(sub, cfg.n, threads=threads)
        out, _ = oracle.decode(np.ascontiguousarray(enc[pos]), pos, cfg.n, cfg.k, threads=threads)
        times.append(time.perf_counter() - t0)
        assert np.array_equal(out, sub)
    t = sum(times) / len(times)
    gbs = cfg.k * cols * 2 / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": cfg.name, "n": cfg.n, "k": cfg.k, "W": cfg.W,
                       "sample_codewords": cols},
            "cpu_baseline": {"value": gbs, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{cols} codewords per step (encode + decode incl. pattern)"},
            "e2e": {"value": gbs, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_0907_1788_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = WORKLOAD
    n, k, W = cfg.n, cfg.k, cfg.W
    stream = torch.cuda.current_stream()
    plan = pkg.Plan(n, k, device=dev)

    # schedules: time every one that can run this workload and keep the fastest
    # (--no-autotune keeps the default schedules, e.g. under a profiler, whose
    # serialised launches would skew the tuner's timings)
    tuned = {}
    for name, op in (("encode", pkg.OP_ENCODE), ("decode", pkg.OP_DECODE)):
        res = [] if args.no_autotune else plan.autotune(W, op, stream)
        tuned[name] = {"timed_us": {pkg.SCHED_NAMES[s_]: round(us, 2) for s_, us in res},
                       "chosen": pkg.SCHED_NAMES[plan.schedule(op)]}

    src = pkg.to_device(cfg.source(), dev)
    enc = torch.empty((n, W), dtype=torch.int32, device=dev)
    out = torch.empty((k, W), dtype=torch.int16, device=dev)
    patterns = [synth.received_positions(n, synth.erased_uniform(cfg.seed * 100 + i, n, k))
                for i in range(N_PATTERNS)]
    # received packets of each pattern, as a receiver holds them (built once)
    pkg.fnt_rs_encode(plan.handle, src, enc, plan.workspace(W, pkg.OP_ENCODE), stream)
    recvs = [torch.index_select(enc, 0, torch.from_numpy(pos.astype(np.int64)).to(dev))
             for pos in patterns]
    # Steady state: source, encoded and decoded buffers rotate over N_SETS copies
    # (with the 8 received matrices: 544 MB touched per rotation, > the 129 MB L2),
    # so nothing a step reads is left in L2 by the step before, and the dirty
    # lines a step leaves are written back during the steps after it, inside
    # their events.
    srcs = [src] + [src.clone() for _ in range(N_SETS - 1)]
    encs = [enc] + [torch.empty_like(enc) for _ in range(N_SETS - 1)]
    outs = [out] + [torch.empty_like(out) for _ in range(N_SETS - 1)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ws_e = plan.workspace(W, pkg.OP_ENCODE)
    ws_d = plan.workspace(W, pkg.OP_DECODE)

    # The decode of a batch needs only its pattern's plan, not this batch's
    # encode, so a step runs plan -> decode on the main stream, which starts at
    # once, and the encode on a second stream that waits for the step's start;
    # the plan kernel thus gets its few SMs before the encode fills the rest,
    # and each of encode and decode fills the other's last wave.
    side = torch.cuda.Stream(device=dev)
    fork, join = torch.cuda.Event(), torch.cuda.Event()

    def step(i, ev=None):
        pos = patterns[i % N_PATTERNS]
        b = i % N_SETS
        if ev:
            ev[0].record(stream)
        fork.record(stream)
        pkg.fnt_rs_decode_prepare(plan.handle, pos, stream)
        side.wait_event(fork)
        pkg.fnt_rs_encode(plan.handle, srcs[b], encs[b], ws_e, side)
        join.record(side)
        pkg.fnt_rs_decode(plan.handle, recvs[i % N_PATTERNS], pos, outs[b], ws_d, stream)
        stream.wait_event(join)
        if ev:
            ev[1].record(stream)

    def round_trip_ok():
        want = cfg.source()
        return all(np.array_equal(pkg.to_host(o), want) for o in outs)

    def step_serial(i, ev):
        # the same work one call after another, to time each phase on its own
        pos = patterns[i % N_PATTERNS]
        b = i % N_SETS
        ev[0].record(stream)
        pkg.fnt_rs_encode(plan.handle, srcs[b], encs[b], ws_e, stream)
        ev[1].record(stream)
        pkg.fnt_rs_decode_prepare(plan.handle, pos, stream)
        ev[2].record(stream)
        pkg.fnt_rs_decode(plan.handle, recvs[i % N_PATTERNS], pos, outs[b], ws_d, stream)
        ev[3].record(stream)

    for i in range(max(args.warmup, N_SETS)):
        step(i)
    torch.cuda.synchronize()
    # correctness of the timed configuration (bit-exact round trip)
    assert round_trip_ok(), "round trip failed"
    assert plan.status() == 0

    # timed region: steps back to back, no flush (buffers rotate, see above)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    launches0 = pkg.fnt_rs_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_wall0 = time.perf_counter()
        for i in range(args.steps):
            step(args.warmup + i, evs[i])
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    launches = pkg.fnt_rs_launch_count() - launches0
    ms_step = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    ms_step = max_over_ranks(ms_step, dev)
    assert round_trip_ok(), "round trip failed (timed)"
    assert plan.status() == 0

    # the same steps with the pattern already in the plan's cache (no build in the
    # step): the difference to the timed step is what the per-pattern build adds
    # to the overlapped step, where it runs beside the encode
    # (4 patterns, the plan's cache holds 4; their received matrices still rotate
    # over 128 MB, so none is read back from L2)
    cev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    for q in range(4):
        pkg.fnt_rs_decode_prepare(plan.handle, patterns[q], stream)
    torch.cuda.synchronize()
    for i in range(args.steps):
        b = i % N_SETS
        cev[i][0].record(stream)
        fork.record(stream)
        side.wait_event(fork)
        pkg.fnt_rs_encode(plan.handle, srcs[b], encs[b], ws_e, side)
        join.record(side)
        pkg.fnt_rs_decode(plan.handle, recvs[i % 4], patterns[i % 4], outs[b], ws_d, stream)
        stream.wait_event(join)
        cev[i][1].record(stream)
    torch.cuda.synchronize()
    ms_cached = sum(e[0].elapsed_time(e[1]) for e in cev) / args.steps
    ms_cached = max_over_ranks(ms_cached, dev)
    assert round_trip_ok(), "round trip failed (cached pattern)"

    # the same steps with L2 flushed before each (the flush outside the events):
    # cold reads, and the write-back of a step's output left outside its events
    fev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_((i + 7) & 0xFF)
        step(args.warmup + i, fev[i])
    torch.cuda.synchronize()
    ms_flushed = sum(e[0].elapsed_time(e[1]) for e in fev) / args.steps
    ms_flushed = max_over_ranks(ms_flushed, dev)
    assert round_trip_ok(), "round trip failed (flushed)"

    # per-phase times (and the dominant kernel's duration for the roofline) from
    # the same steps run serially, back to back over the rotating buffers like
    # the timed steps (each kernel pays the write-back of the dirty lines the
    # kernel before it left in L2); then once more with L2 flushed before each
    # step, where every kernel starts from an L2 full of dirty flush data
    def serial_pass(with_flush, base):
        sev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)]
               for _ in range(args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            if with_flush:
                flush.fill_((i + 3) & 0xFF)
            step_serial(base + i, sev[i])
        torch.cuda.synchronize()
        return ([e[0].elapsed_time(e[1]) for e in sev], [e[1].elapsed_time(e[2]) for e in sev],
                [e[2].elapsed_time(e[3]) for e in sev])

    t_enc, t_pat, t_dec = serial_pass(False, args.warmup + args.steps)
    ms_serial = (sum(t_enc) + sum(t_pat) + sum(t_dec)) / args.steps
    f_enc, f_pat, f_dec = serial_pass(True, args.warmup + 2 * args.steps)
    assert round_trip_ok(), "round trip failed (serial)"

    src_bytes = k * W * 2
    value = whole_job_gbs(src_bytes, world, ms_step)
    enc_ms, pat_ms, dec_ms = (statistics.mean(t_enc), statistics.mean(t_pat),
                              statistics.mean(t_dec))

    # roofline of the dominant kernel: both are integer-issue bound, so the
    # roof is the int32 issue rate; the HBM fraction is reported beside it
    hbm_peak, peak_src = _peaks()
    enc_bytes = W * (2 * k + 4 * n)
    dec_bytes = W * (4 * k + 2 * k) + n * 8 + n * 4
    if dec_ms >= enc_ms:
        dom, dom_ms, dom_bytes, dom_instr = "decode", dec_ms, dec_bytes, W * decode_instr(n, k)
        dom_kernel = "k_decode_tma"
    else:
        dom, dom_ms, dom_bytes, dom_instr = "encode", enc_ms, enc_bytes, W * encode_instr(n, k)
        dom_kernel = "k_encode_tma"
    achieved_tops = dom_instr / (dom_ms * 1e-3) / 1e12
    achieved_gbs = dom_bytes / (dom_ms * 1e-3) / 1e9

    def kernel_roof(ms, nbytes, ninstr):
        tops = ninstr / (ms * 1e-3) / 1e12
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"us": ms * 1e3, "issue_frac": tops / ISSUE_PEAK_TOPS,
                "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak, "bytes_per_launch": nbytes,
                "modelled_instr_per_launch": ninstr}

    per_kernel = {"k_decode_tma": kernel_roof(dec_ms, dec_bytes, W * decode_instr(n, k)),
                  "k_encode_tma": kernel_roof(enc_ms, enc_bytes, W * encode_instr(n, k))}

    # end to end through the host-buffer entry points (pinned memory)
    h_src = torch.from_numpy(cfg.source().view(np.int16)).pin_memory()
    h_enc = torch.empty((n, W), dtype=torch.int32).pin_memory()
    pos0 = patterns[0]
    h_out = torch.empty((k, W), dtype=torch.int16).pin_memory()
    ws_eh = plan.workspace(W, pkg.OP_ENCODE_HOST)
    ws_dh = torch.empty(pkg.fnt_rs_workspace_bytes(plan.handle, W, pkg.OP_DECODE_HOST),
                        dtype=torch.uint8, device=dev)
    pkg.fnt_rs_encode_host(plan.handle, h_src, h_enc, ws_eh, stream)
    h_recv = torch.from_numpy(np.ascontiguousarray(h_enc.numpy()[pos0])).pin_memory()
    e2e_times = []
    for i in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg.fnt_rs_encode_host(plan.handle, h_src, h_enc, ws_eh, stream)
        pkg.fnt_rs_decode_host(plan.handle, h_recv, pos0, h_out, ws_dh, stream)
        e2e_times.append(time.perf_counter() - t0)
    assert np.array_equal(h_out.numpy().view(np.uint16), cfg.source())
    e2e_u32_ms = statistics.median(e2e_times) * 1e3
    e2e_u32 = {"value": world * src_bytes / (e2e_u32_ms * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": k * W * 2 + k * W * 4,
               "d2h_bytes_per_step": n * W * 4 + k * W * 2,
               "format": "32-bit symbols (fnt_rs_encode_host / fnt_rs_decode_host)"}

    # the same round trip in the 16-bit wire format (symbols as 16 bits, the
    # value 65536 as escapes): the public host-buffer calls a sender and a
    # receiver make
    h_enc16 = torch.empty((n, W), dtype=torch.int16).pin_memory()
    h_esc = np.zeros((pkg.fnt_rs_wire_escape_cap(plan.handle, W), 2), dtype=np.uint32)
    ws_ew = plan.workspace(W, pkg.OP_ENCODE_WIRE_HOST)
    ws_dw = torch.empty(pkg.fnt_rs_workspace_bytes(plan.handle, W, pkg.OP_DECODE_WIRE_HOST),
                        dtype=torch.uint8, device=dev)
    nesc = pkg.fnt_rs_encode_wire_host(plan.handle, h_src, h_enc16, h_esc, ws_ew, stream)
    sym16 = h_enc16.numpy().view(np.uint16)
    h_recv16 = torch.from_numpy(np.ascontiguousarray(sym16[pos0]).view(np.int16)).pin_memory()
    r_esc = np.ascontiguousarray(h_esc[:nesc][np.isin(h_esc[:nesc, 0], pos0)])
    rank_of = np.full(n, -1, np.int64)
    rank_of[pos0] = np.arange(len(pos0))
    r_esc[:, 0] = rank_of[r_esc[:, 0]]  # packet -> index of the received row
    e2e_times, e2e_enc = [], []
    for i in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = pkg.fnt_rs_encode_wire_host(plan.handle, h_src, h_enc16, h_esc, ws_ew, stream)
        t1 = time.perf_counter()
        pkg.fnt_rs_decode_wire_host(plan.handle, h_recv16, pos0, r_esc, h_out, ws_dw, stream)
        e2e_times.append(time.perf_counter() - t0)
        e2e_enc.append(t1 - t0)
    assert m == nesc and np.array_equal(h_out.numpy().view(np.uint16), cfg.source())
    e2e_ms = statistics.median(e2e_times) * 1e3
    e2e_enc_ms = statistics.median(e2e_enc) * 1e3
    e2e = {"value": world * src_bytes / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": k * W * 2 + k * W * 2 + len(r_esc) * 8,
           "d2h_bytes_per_step": n * W * 2 + 4 + nesc * 8 + k * W * 2,
           "format": "16-bit wire symbols + escape list (fnt_rs_encode_wire_host / "
                     "fnt_rs_decode_wire_host)",
           "escapes": int(nesc), "ms": e2e_ms, "encode_call_ms": e2e_enc_ms}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": cfg.name, "n": n, "k": k, "W": W, "packet_bytes": 2 * W,
                   "erasures": "uniform, fresh pattern per step (8 cycling > 4 cached)",
                   "step": "(decode plan -> decode of k received packets) || encode, two streams",
                   "l2": (f"not flushed: inputs larger than L2 (source, encoded and decoded "
                          f"buffers rotate over {N_SETS} sets, 8 received matrices; 544 MB "
                          "touched per rotation > 129 MB L2); each step's write-back lands "
                          "inside later steps' events"),
                   "parallelism": f"replicas x{world}"},
        "autotune": tuned,
        "breakdown_ms": {"encode": enc_ms, "plan": pat_ms, "decode": dec_ms,
                         "serial_step": ms_serial,
                         "how": "the step's three calls one after another on one stream, "
                                "back to back over the rotating buffers (no flush); means"},
        "breakdown_flushed_ms": {"encode": statistics.mean(f_enc),
                                 "plan": statistics.mean(f_pat),
                                 "decode": statistics.mean(f_dec),
                                 "how": "the same with a 256 MB L2 flush before each step "
                                        "(the flush's dirty lines are written back during "
                                        "the kernels)"},
        "cached_pattern": {"ms_per_step": ms_cached,
                           "plan_cost_in_step_ms": ms_step - ms_cached,
                           "how": "the same overlapped steps with the pattern already cached "
                                  "(no pattern build in the step)"},
        "flushed": {"ms_per_step": ms_flushed,
                    "value": whole_job_gbs(src_bytes, world, ms_flushed),
                    "how": "the same steps with a 256 MB L2 flush before each, outside the "
                           "events (output write-back left outside the timed region)"},
        "encode_gbs": src_bytes / (enc_ms * 1e-3) / 1e9,
        "decode_gbs": src_bytes / (dec_ms * 1e-3) / 1e9,
        "decode_incl_plan_gbs": src_bytes / ((dec_ms + pat_ms) * 1e-3) / 1e9,
        "roofline": {"bound": "alu", "kernel": dom_kernel, "achieved": achieved_tops,
                     "peak": ISSUE_PEAK_TOPS, "unit": "Tops/s", "frac": achieved_tops / ISSUE_PEAK_TOPS,
                     "traffic": _traffic(dom_kernel),
                     "ops_per_launch": dom_instr,
                     "peak_source": "152 SM x 4 schedulers x 32 lanes x 2070 MHz (int32 issue)",
                     "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                             "frac": achieved_gbs / hbm_peak, "peak_source": peak_src,
                             "bytes_per_launch": dom_bytes},
                     "hbm_frac": achieved_gbs / hbm_peak,
                     "kernels": per_kernel},
        "e2e": e2e,
        "e2e_u32": e2e_u32,
        "bit_exact": {"round_trip": True, "codewords": W,
                      "checked": "decode(encode(s)) == s on every codeword after the timed, "
                                 "serial and end-to-end passes (the run aborts otherwise); "
                                 "oracle parity is the test suite's"},
        "gpu_launches": int(launches),
        "wall_ms_per_step": t_wall * 1e3 / args.steps,
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_extras:
        line["ragged"] = ragged_measure(pkg, dev, max_groups=args.ragged_groups or None)
        sv = serving_sweep(pkg, count=args.serving_requests)
        line["serving"] = sv
        # the serving figures of the metric, at the trace's lowest rate, on one clock
        # (latency from each request's scheduled arrival, queueing included)
        line["serving_p50_ms"] = sv["p50_ms"]
        line["serving_p99_ms"] = sv["p99_ms"]
        line["serving_gbs"] = sv["achieved_gbs"]
        line["serving_baseline_p50_ms"] = sv["baseline"]["p50_ms"]
        line["serving_baseline_p99_ms"] = sv["baseline"]["p99_ms"]
        line["serving_baseline_gbs"] = sv["baseline"]["achieved_gbs"]
        line["systematic"] = systematic_measure(pkg, dev)
        line["wire"] = wire_measure(pkg, dev)
        line["paper_route"] = paper_route_measure(pkg, dev)
        line["direct"] = direct_measure(pkg, dev)
        line["large"] = large_code_measure(pkg, dev)
        line["rates"] = rate_measure(pkg, dev)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the ragged and serving runs")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default schedules instead of timing every candidate")
    ap.add_argument("--ragged-groups", type=int, default=0,
                    help="groups of the seed-4 ragged batch to run (0: all 4096)")
    ap.add_argument("--serving-requests", type=int, default=3000,
                    help="requests replayed per arrival rate in the serving measurement")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
