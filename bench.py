"""Benchmark: FNT-RS encode + per-pattern plan + erasure decode on GB300.

One step = one batch of the k=4096, n=8192, 2048-codeword workload (4 KB
packets, uniform random 16-bit source, one fresh uniform erasure pattern of
n-k positions per batch): encode the batch, build the pattern's decode plan
(steps 1-3), decode every codeword from the k received packets (stacked in
arrival order, the packed layout of the C ABI).

value = source bytes (k * W * 2) round-tripped per second (encode + plan +
decode), summed over ranks.  Per-step CUDA-event times exclude the L2 flush
that separates steps (a 256 MB write).  `--impl reference` times the CPU
oracle on a bounded sample of the same workload.
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


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{index}.csv")

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

    src = pkg.to_device(cfg.source(), dev)
    enc = torch.empty((n, W), dtype=torch.int32, device=dev)
    out = torch.empty((k, W), dtype=torch.int16, device=dev)
    patterns = [synth.received_positions(n, synth.erased_uniform(cfg.seed * 100 + i, n, k))
                for i in range(N_PATTERNS)]
    # received packets of each pattern, as a receiver holds them (built once)
    pkg.fnt_rs_encode(plan.handle, src, enc, plan.workspace(W, pkg.OP_ENCODE), stream)
    recvs = [torch.index_select(enc, 0, torch.from_numpy(pos.astype(np.int64)).to(dev))
             for pos in patterns]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ws_e = plan.workspace(W, pkg.OP_ENCODE)
    ws_d = plan.workspace(W, pkg.OP_DECODE)

    def step(i, ev=None):
        pos = patterns[i % N_PATTERNS]
        if ev:
            ev[0].record(stream)
        pkg.fnt_rs_encode(plan.handle, src, enc, ws_e, stream)
        if ev:
            ev[1].record(stream)
        pkg.fnt_rs_decode_prepare(plan.handle, pos, stream)
        if ev:
            ev[2].record(stream)
        pkg.fnt_rs_decode(plan.handle, recvs[i % N_PATTERNS], pos, out, ws_d, stream)
        if ev:
            ev[3].record(stream)

    for i in range(args.warmup):
        flush.fill_(i & 0xFF)
        step(i)
    torch.cuda.synchronize()
    # correctness of the timed configuration (bit-exact round trip)
    assert np.array_equal(pkg.to_host(out), cfg.source()), "round trip failed"
    assert plan.status() == 0

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    launches0 = pkg.fnt_rs_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_((i + 7) & 0xFF)
            step(args.warmup + i, evs[i])
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    launches = pkg.fnt_rs_launch_count() - launches0
    t_enc = [e[0].elapsed_time(e[1]) for e in evs]
    t_pat = [e[1].elapsed_time(e[2]) for e in evs]
    t_dec = [e[2].elapsed_time(e[3]) for e in evs]
    ms_step = (sum(t_enc) + sum(t_pat) + sum(t_dec)) / args.steps
    if world > 1:
        tt = torch.tensor([ms_step], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_step = float(tt.item())
    assert np.array_equal(pkg.to_host(out), cfg.source()), "round trip failed (timed)"

    src_bytes = k * W * 2
    value = world * src_bytes / (ms_step * 1e-3) / 1e9
    enc_ms, pat_ms, dec_ms = (statistics.mean(t_enc), statistics.mean(t_pat),
                              statistics.mean(t_dec))

    # roofline of the dominant kernel (algorithmic bytes per launch / duration)
    hbm_peak, peak_src = _peaks()
    enc_bytes = W * (2 * k + 4 * n)
    dec_bytes = W * (4 * k + 2 * k) + n * 8 + n * 4
    if dec_ms >= enc_ms:
        dom, dom_ms, dom_bytes = "decode", dec_ms, dec_bytes
    else:
        dom, dom_ms, dom_bytes = "encode", enc_ms, enc_bytes
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9

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
    e2e_ms = statistics.median(e2e_times) * 1e3
    e2e = {"value": world * src_bytes / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": k * W * 2 + k * W * 4,
           "d2h_bytes_per_step": n * W * 4 + k * W * 2}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": cfg.name, "n": n, "k": k, "W": W, "packet_bytes": 2 * W,
                   "erasures": "uniform, fresh pattern per step (8 cycling > 4 cached)",
                   "step": "encode + decode plan + decode (k received packets)",
                   "l2": "flushed between steps (256 MB write, outside the events)",
                   "parallelism": f"replicas x{world}"},
        "breakdown_ms": {"encode": enc_ms, "plan": pat_ms, "decode": dec_ms},
        "encode_gbs": src_bytes / (enc_ms * 1e-3) / 1e9,
        "decode_gbs": src_bytes / (dec_ms * 1e-3) / 1e9,
        "decode_incl_plan_gbs": src_bytes / ((dec_ms + pat_ms) * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak,
                     "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                     "peak_source": peak_src},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "wall_ms_per_step": t_wall * 1e3 / args.steps,
        "clocks": clk.summary(),
    }
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
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
