#!/usr/bin/env python
"""Benchmark: timing arcs per second of the full STA pass on one B300.

A step is one ``sta_update_timing`` (dataflow schedule by default) -- net
delay calculation, forward
arrival/slew propagation, endpoint required times, backward required-time
propagation with pin slacks, and the FP64 WNS/TNS reduction -- over the
seeded 1M-cell synthetic design (depth 150, RC trees of 2-10 nodes, one
corner).  Arcs are counted once per pass (cell arcs + net arcs).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank times its own
replica of the design (replicas only: a single design's levels do not shard)
and ``value`` sums the ranks' arcs over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import collections
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "timing arcs/sec (fwd+bwd STA) and grad ms/iter at 1M cells, batched vs plain"
UNIT = "arcs/s"
WORKLOADS = {
    "scale": "1M cells, depth 150, RC trees of 2-10 nodes, 1 corner, clock period at the 90th percentile "
             "endpoint requirement (seed 0)",
    "mid": "200k cells, depth 150, RC trees of 2-10 nodes, 1 corner (profiler-sized; seed 0)",
    "steiner": "1M cells, depth 150, placed in a 1000 um die, Steiner-tree RC rebuilt from the positions at every "
               "update, 1 corner (seed 0)",
    "steiner_mid": "200k cells, depth 150, placed, Steiner-tree RC from positions (profiler-sized; seed 0)",
    "batch": "64 designs, cells log-uniform in 5k-500k, depth 150, 4 corners, one batched context against 256 "
             "sequential plain passes (seed 0)",
    "large": "10M cells, depth 400, placed in a 1000 um die (star RC), 4 corners, 2 drive strengths, "
             "gamma 0.01 ns; 20 iterations of 1% moves + 1% resizes + timing + gradient (seed 0)",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale", choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--schedule", default="dataflow", choices=["level", "dataflow", "coop", "tile", "auto"],
                    help="propagation schedule; auto = sta_autotune's choice")
    ap.add_argument("--net-model", default="elmore", choices=["elmore", "arnoldi"],
                    help="net delay calculator of the scale/mid workloads (arnoldi: order-3 reduced model)")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the update only (no e2e, CPU baseline, batch, gradient or clock sampling); for profilers")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-plain comparison")
    ap.add_argument("--batch-designs", type=int, default=64)
    ap.add_argument("--batch-hi", type=int, default=500_000, help="largest design of the batch (cells)")
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient timing")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 10M-cell x 4-corner incremental differentiable loop")
    return ap.parse_args()


# --------------------------------------------------------------- helpers

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) > 8:
                for n, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def byte_model(st: dict, K: int) -> dict:
    """Algorithmic (compulsory) bytes of one update per kernel, FP32 pin
    states, each element read once and written once (cache reuse of fan-in
    gathers is not credited).  P pins, A timing arcs (cell + net), S net
    sinks, Nn nets, N RC nodes; K corners multiply the per-pin, per-sink and
    per-net terms.
      net    RC read 12 B/node; load write 4 B/net; sink delay and variance write 8 B/sink
      fwd    arrival + slew write 32 B/pin and read 32 B/pin; fan-in CSR 8 B/arc + offsets 4 B/pin;
             net outputs read (4 B/net, 8 B/sink)
      bwd    required time write + read 32 B/pin; slews re-read 16 B/pin; arrival and required read for
             slack 32 B/pin, slack write 16 B/pin; fan-out CSR 8 B/arc + offsets 4 B/pin
    Total = 168P + 16A + 12N + 16S + 8Nn per corner-scaled term."""
    P, S, Nn, N = st["n_pins"], st["n_net_arcs"], st["n_nets"], st["n_rc_nodes"]
    A = st["n_cell_arcs"] + st["n_net_arcs"]
    net = 12 * N + K * (4 * Nn + 8 * S)
    fwd = K * (64 * P + 4 * P + 4 * Nn + 8 * S) + 8 * A
    bwd = K * (48 * P + 48 * P + 4 * P) + 8 * A
    return {"net": net, "fwd": fwd, "bwd": bwd, "reduce": 0, "total": net + fwd + bwd}


def storage_model(st: dict, K: int) -> dict:
    """Bytes the implementation's own arrays move per update: arrival and
    required times are double-float (32 B per pin and state), slews and
    slacks FP32 (16 B), E endpoints, I items."""
    P, S, Nn, N = st["n_pins"], st["n_net_arcs"], st["n_nets"], st["n_rc_nodes"]
    E, I = st["n_endpoints"], st["n_items"]
    net = 12 * N + 8 * S + K * (4 * Nn + 8 * S)
    fwd = K * (96 * P + 8 * S + 4 * Nn) + 4 * S + 8 * I
    bwd = K * (128 * P + 4 * S + 4 * Nn + 10 * E) + 4 * S + 4 * I
    red = K * 8 * E
    return {"net": net, "fwd": fwd, "bwd": bwd, "reduce": red, "total": net + fwd + bwd + red}


# the source files that define each measured kernel (its code and everything it inlines)
_PERSISTENT = ("dataflow.cu", "item.cuh", "device.cuh", "kernels.h")
_LEVEL = ("kernels.cu", "item.cuh", "device.cuh", "kernels.h")
_TILE = ("tile.cu", "item.cuh", "device.cuh", "kernels.h")
KERNEL_SOURCES = {"k_df_forward": _PERSISTENT, "k_df_backward": _PERSISTENT, "k_coop_pass": _PERSISTENT,
                  "k_net_tree": _LEVEL, "k_fwd_level": _LEVEL, "k_bwd_level": _LEVEL,
                  "k_tile_forward": _TILE, "k_tile_backward": _TILE}


def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2511_11660_b300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.txt),
    if it was taken on the kernel's current sources (else null)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(p).read().splitlines()
    except OSError:
        return None
    if kernel not in KERNEL_SOURCES:
        return None
    for ln in lines:
        f = ln.split()
        if len(f) == 3 and not ln.startswith("#") and f[0] == kernel and f[1] == kernel_source_hash(kernel):
            return float(f[2])
    return None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def make_workload(name: str, seed: int):
    from paper_2511_11660_b300 import synth
    return synth.workload(name, seed=seed)


# ------------------------------------------------------------------ ours

def run_ours(a, dist: Dist):
    import torch
    from paper_2511_11660_b300 import clock, sta, synth

    torch.cuda.set_device(dist.local)
    dev = dist.local
    d = make_workload(a.workload, a.seed)
    if a.net_model == "arnoldi":
        d.update(net_model=sta.NET_ARNOLDI, arnoldi_order=3)
    dstats = synth.design_stats(d)
    ctx = sta.Context(d, device=dev)
    sched_names = {sta.SCHED_LEVEL: "level", sta.SCHED_DATAFLOW: "dataflow", sta.SCHED_COOP: "coop",
                   sta.SCHED_TILE: "tile"}
    if a.schedule == "auto":
        sch, par, _ = ctx.autotune(trials=5)
        schedule = sched_names[sch]
    else:
        schedule = a.schedule
        ctx.set_schedule({v: k for k, v in sched_names.items()}[schedule], 0)
    # clock period: 90th-percentile endpoint requirement from a run at T = 0
    ctx.set_clock(0.0)
    ctx.update_timing()
    s0, _, _, _ = ctx.get_endpoint_slack()
    T, half_gap = clock.period_in_gap(-s0[:, 0])
    ctx.set_clock(T)
    st = ctx.stats()
    K = st["n_corners"]
    arcs = dstats["arcs"]
    stream = torch.cuda.current_stream()

    for _ in range(a.warmup):
        ctx.update_timing()
    torch.cuda.synchronize()

    sampler = ClockSampler(dev) if not a.no_extras else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        ctx.update_timing()
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    ms_total = e0.elapsed_time(e1)
    clocks = sampler.stop() if sampler else None
    ms_step = dist.max(ms_total) / a.steps
    value = arcs * dist.world / (ms_step * 1e-3)
    rep = ctx.report_slack()[0]

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "%s: %s" % (a.workload, WORKLOADS[a.workload]),
                      "cells": dstats["cells"], "pins": dstats["pins"], "cell_arcs": dstats["cell_arcs"],
                      "net_arcs": dstats["net_arcs"], "rc_nodes": dstats["rc_nodes"],
                      "endpoints": dstats["endpoints"], "levels": st["n_levels"], "corners": K,
                      "period_ns": T, "schedule": schedule, "net_model": a.net_model,
                      "parallelism": "replicas x%d" % dist.world if dist.world > 1 else "1 GPU",
                      "l2": "no flush: per-pass working set %.0f MB > 126 MB L2" % (st["device_bytes"] / 1e6),
                      "wns_setup_ns": rep["wns_setup"], "tns_setup_ns": rep["tns_setup"],
                      "setup_violations": rep["n_viol_setup"]},
           "gpu_launches": st["launches_per_update"] * a.steps}

    if a.no_extras:
        if dist.rank == 0:
            print(json.dumps(out))
        return

    # ---- roofline of the dominant kernel, from per-phase CUDA events
    ctx.set_profiling(True)
    acc = np.zeros(4)
    n_prof = 5
    for _ in range(n_prof):
        ctx.update_timing()
        ctx.sync()
        acc += np.array(ctx.last_timings())
    ctx.set_profiling(False)
    ph = acc / n_prof
    bm = byte_model(st, K)
    pk, pk_kind = peaks()
    fwd_dominant = ph[1] >= ph[2]
    phase_ms = ph[1] if fwd_dominant else ph[2]
    phase_bytes = bm["fwd"] if fwd_dominant else bm["bwd"]
    if schedule == "dataflow":
        kern = "k_df_forward" if fwd_dominant else "k_df_backward"
        launches = 1
    elif schedule == "tile":
        kern = "k_tile_forward" if fwd_dominant else "k_tile_backward"
        launches = 1
    elif schedule == "coop":
        # one launch runs both passes: its time is the forward slot
        kern, launches = "k_coop_pass", 1
        phase_ms, phase_bytes = ph[1] + ph[2], bm["fwd"] + bm["bwd"]
    else:
        kern = "k_fwd_level" if fwd_dominant else "k_bwd_level"
        launches = st["n_levels"]
    achieved = phase_bytes / (phase_ms * 1e-3) / 1e9
    tr = measured_traffic(kern)
    sm = storage_model(st, K)
    if schedule == "coop":
        storage = sm["fwd"] + sm["bwd"]
    else:
        storage = sm["fwd"] if fwd_dominant else sm["bwd"]
    out["roofline"] = {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": pk["hbm_gbs"],
                       "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                       "traffic": tr, "peak_source": pk_kind + " (hbm_gbs, copy burst)",
                       "bytes_per_launch": phase_bytes / launches, "launches_per_pass": launches,
                       "byte_model": "algorithmic: 168P + 16A + 12N + 16S + 8Nn per pass, split per kernel",
                       "storage_bytes_per_launch": storage / launches,
                       "phase_ms": {"net": ph[0], "fwd": ph[1], "bwd": ph[2], "reduce": ph[3]},
                       "pass_bytes_model": bm["total"], "pass_storage_bytes": sm["total"],
                       "pass_frac": bm["total"] / (ms_step * 1e-3) / 1e9 / pk["hbm_gbs"]}

    # ---- end to end through the C ABI with host buffers
    if d.get("rc_R") is not None:
        # two page-locked R/C sets staged in turn on a copy stream: the copy of
        # step i + 1's parasitics runs while step i's update computes
        rc_sets = [(torch.from_numpy(np.asarray(d["rc_R"], np.float32)).pin_memory(),
                    torch.from_numpy(np.asarray(d["rc_C"], np.float32)).pin_memory()) for _ in range(2)]
        h2d = rc_sets[0][0].numel() * 4 + rc_sets[0][1].numel() * 4
        copy_stream = torch.cuda.Stream()
        feed_i = [0]

        def feed():
            Rh, Ch = rc_sets[feed_i[0] & 1]
            ctx.set_rc_async(Rh, Ch, stream=copy_stream)
            feed_i[0] += 1
    else:
        XY = torch.from_numpy(np.asarray(d["cell_xy"], np.float32)).pin_memory()
        h2d = XY.numel() * 4
        feed = lambda: ctx.set_positions(XY)  # noqa: E731
    E = st["n_endpoints"]
    # page-locked host buffers for the endpoint results (direct DMA)
    pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory().numpy()  # noqa: E731
    ep_out = (pin((E, K), torch.float32), pin((E, K), torch.float32), pin((E, K), torch.uint8),
              pin((E, K), torch.uint8))
    # each step: the update, the host-to-device copy of the next step's
    # inputs (overlapping the update where the API allows it), the
    # endpoint results back to the host
    feed()
    for _ in range(2):
        ctx.update_timing(); feed(); ctx.get_endpoint_slack(out=ep_out); ctx.report_slack()
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        ctx.update_timing()
        feed()
        ctx.get_endpoint_slack(out=ep_out)
        ctx.report_slack()
    torch.cuda.synchronize()
    t_e2e = dist.max(time.perf_counter() - t0) / a.steps
    out["e2e"] = {"value": arcs * dist.world / t_e2e, "unit": UNIT,
                  "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(E * K * 10 + 64 * K),
                  "ms_per_step": t_e2e * 1e3,
                  "what": "per step: sta_update_timing, sta_set_rc_async of the next step's R/C from "
                          "pinned host memory on a copy stream (overlapping the update), endpoint slacks and "
                          "violation flags to pinned host buffers, sta_report_slack"}

    # ---- top-k path report (1000 worst endpoints' critical paths, host arrays)
    ctx.report_paths(1000)
    t0 = time.perf_counter()
    n_rep = 5
    for _ in range(n_rep):
        paths = ctx.report_paths(1000)
    out["paths"] = {"k": 1000, "ms_per_report": (time.perf_counter() - t0) / n_rep * 1e3,
                    "pins": int(sum(len(p["pins"]) for p in paths)),
                    "what": "sta_report_paths: radix select of the 1000 worst setup endpoints, bitonic sort, "
                            "critical-path trace, CSR arrays copied to the host"}
    ctx.report_paths(1000, per_endpoint=4)
    t0 = time.perf_counter()
    for _ in range(n_rep):
        paths = ctx.report_paths(1000, per_endpoint=4)
    out["paths"]["per_endpoint_4"] = {
        "ms_per_report": (time.perf_counter() - t0) / n_rep * 1e3, "paths": len(paths),
        "endpoints": len({p["endpoint"] for p in paths}),
        "what": "sta_report_paths_nworst: the 1000 worst paths, at most 4 per endpoint (best-first deviation "
                "search per selected endpoint, merge by slack), CSR arrays copied to the host"}

    # ---- timing exceptions: three startpoint groups with up to two -through
    # sets of 1/64 of the gate inputs each (one tag per group stage)
    if d.get("exc_action") is None:
        dx = dict(d, **synth.exception_groups(d, np.random.default_rng(a.seed), 3, div_from=5, div_to=4, max_thru=2,
                                              div_thru=64))
        dx["period_ns"] = T
        del ctx
        torch.cuda.empty_cache()
        ctx = sta.Context(dx, device=dev)
        # eight states per pin: the schedule comes from sta_autotune (the
        # cooperative one wins here, the dataflow one on a single state)
        sch_x, par_x, _ = ctx.autotune(force=True)
        for _ in range(3):
            ctx.update_timing()
        ms = _events_ms(ctx.update_timing, 10)
        ctx.set_schedule({v: k for k, v in sched_names.items()}[schedule], 0)
        for _ in range(2):
            ctx.update_timing()
        ms_same = _events_ms(ctx.update_timing, 10)
        rx = ctx.report_slack()[0]
        out["exceptions"] = {"groups": 3, "states_per_pin": ctx.stats()["n_tags"] * K, "ms_per_update": ms,
                             "arcs_per_s": arcs / (ms * 1e-3), "schedule": "%s (%d)" % (sched_names[sch_x], par_x),
                             "ms_per_update_%s" % schedule: ms_same, "wns_setup_ns": rx["wns_setup"],
                             "setup_violations": rx["n_viol_setup"],
                             "what": "sta_update_timing with 3 false-path / multicycle groups (1/5 of the "
                                     "startpoints each, 0-2 ordered -through sets of 1/64 of the gate inputs, "
                                     "endpoint lists of 1/4 of the endpoints or all), schedule from sta_autotune"}

    # ---- Steiner-tree RC from positions: a placed 1M-cell design, trees rebuilt every update
    del ctx
    torch.cuda.empty_cache()
    ds = synth.workload("steiner", seed=a.seed)
    ctx = sta.Context(ds, device=dev)
    ctx.set_schedule({v: k for k, v in sched_names.items()}[schedule], 0)
    ctx.set_clock(0.0)
    ctx.update_timing()
    s0, _, _, _ = ctx.get_endpoint_slack()
    ctx.set_clock(clock.period_in_gap(-s0[:, 0], min_half_gap=0.0)[0])
    for _ in range(3):
        ctx.update_timing()
    ms = _events_ms(ctx.update_timing, 10)
    ctx.set_profiling(True)
    acc = np.zeros(4)
    for _ in range(5):
        ctx.update_timing()
        ctx.sync()
        acc += np.array(ctx.last_timings())
    ctx.set_profiling(False)
    wl = ctx.get_net_wirelength()
    sst = synth.design_stats(ds)
    out["steiner"] = {"cells": ds["n_cells"], "nets": ds["n_nets"], "ms_per_update": ms,
                      "arcs_per_s": sst["arcs"] / (ms * 1e-3), "net_phase_ms": acc[0] / 5,
                      "total_wirelength_m": float(wl.sum()) * 1e-9,
                      "what": "sta_update_timing on the steiner workload (1M cells placed locally, "
                              "STA_WIRE_STEINER): Steiner trees of every net from the positions, RC sweep, forward, "
                              "backward, reduction"}

    del ctx
    torch.cuda.empty_cache()
    if not a.no_grad:
        out["grad"] = run_grad(a, dev)
    if not a.no_batch:
        out["batched"] = run_batched(a, dev)
    if not a.no_large:
        out["large"] = incremental_loop(a, dev)

    # ---- the FP64 oracle on the host cores (rank 0, one GPU only)
    if dist.rank == 0 and dist.world == 1:
        out["cpu_baseline"] = cpu_baseline(d, T)
    if clocks is not None:
        out["clocks"] = clocks
    if dist.rank == 0:
        print(json.dumps(out))


def _events_ms(fn, n: int) -> float:
    import torch
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(n):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def run_grad(a, dev: int) -> dict:
    """ms per gradient iteration = sta_set_positions (device) + sta_update_timing
    + sta_backward (device outputs), on placed designs with gamma = 0.01 ns."""
    import torch
    from paper_2511_11660_b300 import clock, sta, synth
    res = {}
    for name, d in (("diff_200k", synth.workload("diff", seed=a.seed)),
                    ("placed_1M", synth.make_design(1_000_000, 150, seed=a.seed, rc_nodes=(2, 10), placed=True,
                                                    gamma_ns=0.01)),
                    ("steiner_1M", dict(synth.workload("steiner", seed=a.seed), gamma_ns=0.01))):
        ctx = sta.Context(d, device=dev)
        ctx.set_schedule(sta.SCHED_DATAFLOW, 0)
        ctx.set_clock(0.0)
        ctx.update_timing()
        s0, _, _, _ = ctx.get_endpoint_slack()
        ctx.set_clock(clock.period_in_gap(-s0[:, 0], min_half_gap=0.0)[0])
        xy = torch.tensor(np.asarray(d["cell_xy"], np.float32), device="cuda")
        grad = torch.empty((d["n_cells"], 2), dtype=torch.float64, device="cuda")

        def it():
            ctx.set_positions(xy)
            ctx.update_timing()
            ctx.backward(1.0, 1.0, grad_out=grad)
        for _ in range(3):
            it()
        ms = _events_ms(it, 10)
        res[name] = {"ms_per_iter": ms, "cells": d["n_cells"], "pins": d["n_pins"],
                     "what": "set_positions + update_timing (dataflow) + sta_backward, all on the device" +
                             ("; Steiner trees rebuilt every iteration, gradient through the trees held fixed"
                              if d.get("wire_model") == 1 else "")}
        ctx.close()
    return res


def run_batched(a, dev: int, plain: bool = True, dist: Dist = None) -> dict:
    """One batched context (64 designs, cells log-uniform in 5k-500k, depth
    150, 4 corners) against 256 sequential plain passes (one design, one
    corner each), device time.  Under torchrun the designs are split over
    the ranks (longest-processing-time on arcs); each rank times a batched
    context of its own share and the per-design reports are gathered on the
    host."""
    from paper_2511_11660_b300 import shard, sta, synth
    ds = synth.batch_workload(seed=a.seed, n_designs=a.batch_designs, hi=a.batch_hi)
    part = list(range(len(ds)))
    if dist is not None and dist.world > 1:
        part = shard.lpt_partition([synth.design_stats(d)["arcs"] for d in ds], dist.world)[dist.rank]
        ds = [ds[i] for i in part]
    arcs = sum(synth.design_stats(d)["arcs"] for d in ds)
    K = ds[0]["n_corners"]
    names = {sta.SCHED_LEVEL: "level", sta.SCHED_DATAFLOW: "dataflow", sta.SCHED_COOP: "coop", sta.SCHED_TILE: "tile"}
    b = sta.Context(None, batch=ds, device=dev)
    sch, par, _ = b.autotune(trials=3)
    for _ in range(3):
        b.update_timing()
    if dist is not None:
        dist.barrier()
    ms_batch = _events_ms(b.update_timing, 10)
    reports = {i: [(r["wns_setup"], r["tns_setup"]) for r in b.report_slack(j)] for j, i in enumerate(part)}
    if dist is not None and dist.world > 1:
        reports = shard.gather_reports(reports, dist.pg)
        ms_batch = dist.max(ms_batch)
        arcs = int(dist.sum(arcs))
    b.close()
    del b
    ls, rs = synth.lut_corners()
    ms_plain = 0.0
    plain_sched = collections.Counter()
    for d in (ds if plain else []):
        d1 = dict(d)
        d1.update(n_corners=1, lut_scale=np.array([ls[0]], np.float32), rc_scale=np.array([rs[0]], np.float32))
        c = sta.Context(d1, device=dev)
        plain_sched[names[c.autotune(trials=2)[0]]] += 1   # each plain pass on its own best schedule
        for k in range(K):
            c.set_corners([ls[k]], [rs[k]])
            c.update_timing()
            ms_plain += _events_ms(c.update_timing, 3)
        c.close()
    return {"designs": len(ds), "corners": K, "cells": int(sum(d["n_cells"] for d in ds)), "arcs": int(arcs),
            "batched_ms_per_pass": ms_batch, "plain_ms_256_passes": ms_plain,
            "batched_arcs_corners_per_s": arcs * K / (ms_batch * 1e-3),
            "plain_arcs_corners_per_s": arcs * K / (ms_plain * 1e-3) if plain else None,
            "speedup": ms_plain / ms_batch if plain else None, "designs_reported": len(reports),
            "batched_schedule": "%s (%d)" % (names[sch], par), "plain_schedules": dict(plain_sched),
            "what": "device time of one update of the batched context (schedule from sta_autotune) vs the sum of "
                    "256 plain single-design single-corner updates, each context on its own autotuned schedule"}


def run_batch_only(a, dist: Dist):
    import torch
    torch.cuda.set_device(dist.local)
    r = run_batched(a, dist.local, plain=not a.no_extras and dist.world == 1, dist=dist)
    v = r["batched_arcs_corners_per_s"]
    out = {"metric": "arc-corners/s, batched designs x corners in one launch sequence", "value": v,
           "unit": "arc-corners/s", "n_gpus": dist.world, "steps": 10, "warmup": 3,
           "ms_per_step": r["batched_ms_per_pass"], "higher_is_better": True,
           "scaling": "strong" if dist.world > 1 else "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "batch: %d designs, cells log-uniform in 5k-%d, depth 150, 4 corners"
                                  % (a.batch_designs, a.batch_hi),
                      "parallelism": "designs sharded over %d ranks" % dist.world if dist.world > 1 else "1 GPU"},
           "batched": r}
    if dist.rank == 0:
        print(json.dumps(out))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_baseline(d: dict, T: float) -> dict:
    """The FP64 oracle on the host cores: net delays through WNS/TNS timed
    inside the oracle (validation, topological order and levels prepared
    once, outside), median of 3 runs, single-threaded and with OpenMP over
    the pins of a level on every host core."""
    import oracle
    from paper_2511_11660_b300 import synth
    dd = dict(d)
    dd["period_ns"] = T
    arcs = synth.design_stats(d)["arcs"]
    nc = host_cores()
    s1, _ = oracle.sta_timed(dd, 1, 3)
    sn, _ = oracle.sta_timed(dd, nc, 3)
    m1, mn = float(np.median(s1)), float(np.median(sn))
    return {"value": arcs / mn, "unit": UNIT, "cores": nc, "kind": "oracle",
            "sample": "the full workload design, FP64 oracle (gcc -O3), net delays through WNS/TNS timed (order and "
                      "levels prepared outside), median of 3 runs on %d threads (OpenMP over each level's pins): "
                      "%.3f s per pass" % (nc, mn),
            "single_thread": {"value": arcs / m1, "cores": 1, "s_per_pass": m1,
                              "runs_s": [round(float(x), 4) for x in s1]},
            "multi_thread": {"value": arcs / mn, "cores": nc, "s_per_pass": mn,
                             "runs_s": [round(float(x), 4) for x in sn]}}


# ---------------------------------------------------------- incremental

def incremental_loop(a, dev: int, n_iter: int = 20) -> dict:
    """The large incremental differentiable loop on 10M cells x 4 corners:
    per iteration move 1% of the cells by U(-5, 5) um and resize 1% to the
    other drive strength, then set_positions + resize_cells + update_timing
    + sta_backward, all on the device.  Returns ms per iteration (wall and
    device), per-call times and the memory the context holds."""
    import torch
    from paper_2511_11660_b300 import clock, sta, synth
    t0 = time.perf_counter()
    d = make_workload("large", a.seed)
    t_gen = time.perf_counter() - t0
    st_d = synth.design_stats(d)
    t0 = time.perf_counter()
    ctx = sta.Context(d, device=dev)
    t_create = time.perf_counter() - t0
    ctx.set_clock(0.0)
    ctx.update_timing()
    s0, _, _, _ = ctx.get_endpoint_slack()
    T = clock.period_in_gap(-s0[:, 1], min_half_gap=0.0)[0]   # corner 1 (scale 1.0)
    ctx.set_clock(T)
    names = {sta.SCHED_LEVEL: "level", sta.SCHED_DATAFLOW: "dataflow", sta.SCHED_COOP: "coop", sta.SCHED_TILE: "tile"}
    sch, par, _ = ctx.autotune(trials=1)
    K = ctx.K
    C = d["n_cells"]
    rng = np.random.default_rng(a.seed)
    xy = torch.tensor(np.asarray(d["cell_xy"], np.float32), device="cuda")
    types = np.asarray(d["cell_type"], np.int32).copy()
    grad = torch.empty((C, 2), dtype=torch.float64, device="cuda")
    walls, devs = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rz_d = ty_d = None
    for it in range(n_iter + 2):
        mv = torch.from_numpy(rng.choice(C, C // 100, replace=False)).cuda()
        dxy = torch.from_numpy(rng.uniform(-5, 5, size=(C // 100, 2)).astype(np.float32)).cuda()
        xy.view(-1, 2)[mv] += dxy
        rz = rng.choice(C, C // 100, replace=False)
        types[rz] = np.where(types[rz] < 8, types[rz] + 8, types[rz] - 8)
        rz_d = torch.from_numpy(rz.astype(np.int32)).cuda()
        ty_d = torch.from_numpy(types[rz]).cuda()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        e0.record()
        ctx.set_positions(xy)
        ctx.resize_cells(rz_d, ty_d)
        ctx.update_timing()
        J, _, _ = ctx.backward(1.0, 1.0, grad_out=grad)
        e1.record()
        torch.cuda.synchronize()
        if it >= 2:
            walls.append(time.perf_counter() - w0)
            devs.append(e0.elapsed_time(e1))
    # one more iteration, each call timed on its own
    parts = {}
    for name, fn in (("set_positions", lambda: ctx.set_positions(xy)),
                     ("resize_cells", lambda: ctx.resize_cells(rz_d, ty_d)),
                     ("update_timing", lambda: ctx.update_timing()),
                     ("backward", lambda: ctx.backward(1.0, 1.0, grad_out=grad))):
        parts[name] = _events_ms(fn, 1)
    stats = ctx.stats()
    rep = ctx.report_slack()
    ctx.close()
    del ctx
    torch.cuda.empty_cache()
    return {"ms_per_iter": float(np.median(walls) * 1e3), "device_ms_per_iter": float(np.median(devs)),
            "iterations": n_iter, "ms_by_call": parts, "cells": st_d["cells"], "pins": st_d["pins"],
            "arcs": st_d["arcs"], "corners": K, "levels": stats["n_levels"], "period_ns": T,
            "schedule": "%s (%d)" % (names[sch], par), "device_bytes": stats["device_bytes"],
            "generate_s": t_gen, "create_s": t_create,
            "arc_corners_per_s": st_d["arcs"] * K / np.median(walls),
            "wns_setup_ns_by_corner": [r["wns_setup"] for r in rep],
            "gpu_launches_per_iter": stats["launches_per_update"] + stats["launches_per_backward"] + 2,
            "what": "per iteration: 1%% of the cells moved by U(-5, 5) um and 1%% resized (LUTs x0.7), then "
                    "set_positions + resize_cells + update_timing + sta_backward (gamma 0.01 ns), all on the "
                    "device; median of %d iterations after 2 warm-up" % n_iter}


def run_incremental(a, dist: Dist):
    """--workload large: the incremental loop as its own JSON line."""
    import torch
    torch.cuda.set_device(dist.local)
    r = incremental_loop(a, dist.local)
    out = {"metric": "grad ms/iter, incremental differentiable STA (10M cells, 4 corners)",
           "value": r["ms_per_iter"], "unit": "ms/iter", "n_gpus": 1, "steps": r["iterations"], "warmup": 2,
           "ms_per_step": r["ms_per_iter"], "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "large: " + WORKLOADS["large"], "cells": r["cells"], "pins": r["pins"],
                      "arcs": r["arcs"], "corners": r["corners"], "levels": r["levels"],
                      "period_ns": r["period_ns"], "schedule": r["schedule"], "device_bytes": r["device_bytes"],
                      "generate_s": r["generate_s"], "create_s": r["create_s"],
                      "wns_setup_ns_by_corner": r["wns_setup_ns_by_corner"]},
           "device_ms_per_iter": r["device_ms_per_iter"], "ms_by_call": r["ms_by_call"],
           "arc_corners_per_s": r["arc_corners_per_s"],
           "gpu_launches": r["iterations"] * r["gpu_launches_per_iter"]}
    print(json.dumps(out))


# ------------------------------------------------------------- reference

def run_reference(a, dist: Dist):
    """The FP64 oracle timed on the host cores on this arm's workload: each
    step one full analysis (net delays through WNS/TNS, OpenMP over each
    level's pins on every host core; validation and the topological order
    prepared once, outside)."""
    if dist.rank != 0:
        return
    from paper_2511_11660_b300 import synth
    import oracle
    d = make_workload(a.workload, a.seed)
    arcs = synth.design_stats(d)["arcs"]
    nc = host_cores()
    if a.warmup > 0:
        oracle.sta_timed(d, nc, a.warmup)
    secs, _ = oracle.sta_timed(d, nc, a.steps)
    t = float(np.mean(secs))
    v = arcs / t
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": dist.world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "%s: %s" % (a.workload, WORKLOADS[a.workload]), "arcs": arcs},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": nc, "kind": "oracle",
                            "sample": "one full oracle analysis of the workload design per step, %d threads" % nc},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    a = parse()
    dist = Dist()
    try:
        if a.impl == "reference":
            run_reference(a, dist)
        elif a.workload == "large":
            run_incremental(a, dist)
        elif a.workload == "batch":
            run_batch_only(a, dist)
        else:
            run_ours(a, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
