#!/usr/bin/env python
"""Throughput of exact O(mM) belief propagation on a GB300.

Metric: message updates per second (directed edges x labels x iterations per
second) of the O(mM) sum-product update (Eq. 7) on the 1280 x 720, M = 128,
T = 4 random-dot stereo workload, 100 synchronous iterations per step, plus the
O(M^2) baselines on the same grid and their fraction of the HBM roofline.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

One JSON line on stdout (rank 0).  N > 1 (torchrun) runs independent replicas,
one per GPU (the grid update has no exchange step here), and reports the
aggregate over ranks with the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1010_0012_gb300 import workload as wl  # noqa: E402

METRIC = "message updates/s (edges*labels/s), O(mM) band update"
UNIT = "updates/s"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid1280x720_m128")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-throughput", action="store_true",
                    help="skip the FP32 O(mM) vs O(M^2) comparison on the host cores")
    ap.add_argument("--no-baselines", action="store_true", help="skip the O(M^2) baselines")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 384x288, 64-MRF batch and gradient workloads in the default line")
    ap.add_argument("--persistent", type=int, default=-1, choices=[-1, 0, 1],
                    help="issue form of single-grid iterations (see bp_set_persistent)")
    ap.add_argument("--rows", type=int, default=0,
                    help="use only this many image rows (smaller case for profiling)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    return {"hbm_gbs": FALLBACK_HBM_GBS, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "source": "fallback"}


def recorded_traffic(kernel, cfg):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the kernel source as it stands now (else None)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p) or cfg.name != "grid1280x720_m128" or cfg.H != 720:
        return None
    rec = json.load(open(p)).get(kernel)
    if not rec:
        return None
    h = hashlib.sha256()
    for f in rec["source_files"]:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return rec["dram_bytes_full_launch"] if h.hexdigest() == rec["source_sha256"] else None


def workload_units(cfg):
    De = wl.directed_edges(cfg.W, cfg.H)
    return De * cfg.M          # message updates per iteration


def algorithmic_bytes(cfg, elem=4):
    """Bytes one synchronous iteration must move: read the unary and every
    incoming message, write every outgoing message."""
    De = wl.directed_edges(cfg.W, cfg.H)
    return (cfg.W * cfg.H * cfg.M + 2 * De * cfg.M) * elem


# ------------------------------------------------------------ clock sampler ----

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_ready(self, timeout=3.0):
        """Block until the first sample arrives: nvidia-smi's start-up (driver
        and NVML initialisation) then falls outside the timed region, where it
        could stall the host's CUDA calls of a wall-clock measurement."""
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons, pw = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            try:
                pw.append(float(f[3]))
            except ValueError:
                pass
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                "power_w": statistics.median(pw) if pw else None}


# --------------------------------------------------------------- CPU oracle ----

def oracle_sample(cfg, stereo_obj, target_s=10.0):
    """Time the oracle (dense FP64, one thread) on a band of rows of the
    workload: one synchronous iteration.  Returns (updates/s, description)."""
    import oracle
    from oracle import grid, stereo
    g64 = wl.unary_f32(stereo_obj).astype(np.float64)
    tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
    F = stereo.compatibility_matrix(tab.astype(np.float64), cfg.T, fbar, cfg.M)

    def run(rows):
        sub = np.ascontiguousarray(g64[:rows])
        t0 = time.perf_counter()
        grid.grid_sum_product(sub, F, 1, "sync")
        return time.perf_counter() - t0, wl.directed_edges(cfg.W, rows) * cfg.M

    rows = 2
    t, u = run(rows)
    rows = int(max(2, min(cfg.H, rows * target_s / max(t, 1e-3))))
    t, u = run(rows)
    return u / t, f"1 synchronous iteration on rows 0..{rows - 1} ({cfg.W}x{rows} grid) of the workload", t


def cpu_throughput_sample(cfg, stereo_obj, rows=180, reps=3):
    """Sec. 6's CPU comparison on this machine's host cores: one FP32
    synchronous iteration of the O(mM) update (Eq. 7) and of the O(M^2)
    update (Eq. 2), OpenMP over rows, on the first `rows` rows of the
    workload (median of `reps` after one warm-up)."""
    import cpu_baselines as cb
    from oracle import stereo
    R = max(2, min(rows, cfg.H))
    g = np.ascontiguousarray(wl.unary_f32(stereo_obj)[:R])
    tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
    F = stereo.compatibility_matrix(tab.astype(np.float64), cfg.T, fbar, cfg.M).astype(np.float32)
    pin = np.full((4, R, cfg.W, cfg.M), 1.0 / cfg.M, np.float32)
    pout = np.empty_like(pin)
    units = wl.directed_edges(cfg.W, R) * cfg.M

    def timed(fn):
        ts = []
        for i in range(reps + 1):
            t0 = time.perf_counter()
            fn()
            if i:
                ts.append(time.perf_counter() - t0)
        return statistics.median(ts)

    tb = timed(lambda: cb.band_iteration(g, pin, pout, tab, cfg.T, fbar))
    td = timed(lambda: cb.dense_iteration(g, pin, pout, F))
    return {"band_mM": {"value": units / tb, "unit": UNIT, "ms_per_iter": 1e3 * tb},
            "dense_M2": {"value": units / td, "unit": UNIT, "ms_per_iter": 1e3 * td},
            "speedup": td / tb, "cores": cb.threads(), "dtype": "f32",
            "sample": f"1 synchronous iteration on rows 0..{R - 1} ({cfg.W}x{R} grid) of the workload, "
                      f"median of {reps}"}


# Algorithmic HBM bytes per message update of each update kind: read the unary
# and the four incoming messages, write the four outgoing ones (9 bytes at
# FP32); the packed tensor-core form also writes its BF16 h rows (8 bytes per
# node-label) and reads them back in the GEMM: 7 + 6 = 13 bytes per update.
UPDATE_BYTES = {"band_mM": 9.0, "dense_bf16_tcgen05_fused": 9.0, "dense_bf16_tcgen05": 13.0,
                "dense_fp32_cuda_core": 9.0}


def time_updates_median(G, stream, cfg, dev, kinds, reps=5):
    """Per-iteration time of each update kind on the handle's grid: one
    warm-up call, then `reps` timed calls of n iterations each (CUDA events on
    the handle's stream), median of the repetitions."""
    import torch
    from paper_1010_0012_gb300 import bp
    pk = peaks()
    units = workload_units(cfg)
    res = {}
    with ClockSampler(dev) as clk:
        clk.wait_ready()
        for name, kind in kinds:
            n_it = 3 if kind == bp.BP_DENSE_CUDA_CORE else 20
            if kind is None:
                fn = (lambda k: (lambda: G.iterate(k, bp.BP_SUM, "sync")))(n_it)
            else:
                fn = (lambda k, n: (lambda: bp.bp_iterate_dense(G.h, n, k)))(kind, n_it)
            try:
                G.reset()
                G.iterate(0, bp.BP_SUM, "sync")
                fn()
                G.sync()
                ts = []
                for _ in range(reps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    fn()
                    b.record(stream)
                    b.synchronize()
                    ts.append(a.elapsed_time(b) / 1e3 / n_it)
                G.sync()
                t = statistics.median(ts)
                ach = units * UPDATE_BYTES[name] / t / 1e9
                res[name] = {"value": units / t, "unit": UNIT, "ms_per_iter": t * 1e3,
                             "ms_per_iter_min_max": [min(ts) * 1e3, max(ts) * 1e3],
                             "timing": f"median of {reps} repetitions of {n_it} iterations (CUDA events)",
                             "roofline": {"bound": "hbm", "bytes_per_update": UPDATE_BYTES[name], "achieved": ach,
                                          "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                                          "peak_source": pk["source"]}}
            except bp.BPError as e:
                res[name] = {"unavailable": str(e)[:160]}
    res["clocks"] = clk.summary()
    if "value" in res.get("band_mM", {}) and "value" in res.get("dense_bf16_tcgen05_fused", {}):
        res["band_over_fused_tcgen05"] = res["band_mM"]["value"] / res["dense_bf16_tcgen05_fused"]["value"]
    return res


# ------------------------------------------------------------------ GPU arm ----

def aggregate_over_ranks(elapsed_s, units_local, world, device=None):
    """Whole-job numbers for N independent replicas: the slowest rank's time
    and the units of all ranks (every rank returns the same pair)."""
    if world <= 1:
        return elapsed_s, units_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_ours(args, cfg, rank, world):
    import torch
    from paper_1010_0012_gb300 import bp

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    st = wl.make_stereo(cfg)
    g_host = torch.from_numpy(wl.unary_f32(st)).pin_memory()
    g_dev = g_host.to("cuda")
    tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    G = bp.BPGrid(cfg.W, cfg.H, cfg.M, bp.BP_F32, stream=stream)
    G.set_unary(g_dev)
    G.set_potential(tab, cfg.T, fbar)
    K = cfg.iters
    units_step = workload_units(cfg) * K
    bel = torch.empty((cfg.H, cfg.W, cfg.M), dtype=torch.float32, device="cuda")
    mp = torch.empty((cfg.H, cfg.W), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()      # the handle's stream does not wait on torch's

    def step(ev_pair=None):
        G.reset()
        G.iterate(0, bp.BP_SUM, "sync")      # materialise the uniform start state
        if ev_pair is not None:
            ev_pair[0].record(stream)
        G.iterate(K, bp.BP_SUM, "sync")
        if ev_pair is not None:
            ev_pair[1].record(stream)
        bp.bp_beliefs(G.h, bel, mp)

    for _ in range(args.warmup):
        step()
    G.sync()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    launches0 = G.launches
    with ClockSampler(dev) as clk:
        clk.wait_ready()
        t0.record(stream)
        for i in range(args.steps):
            step(ev[i])
        t1.record(stream)
        t1.synchronize()
    G.sync()
    launches = G.launches - launches0
    elapsed = t0.elapsed_time(t1) / 1e3
    band_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    elapsed, units_all = aggregate_over_ranks(elapsed, units_step * args.steps, world, device="cuda")
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    out = {"elapsed": elapsed, "units": units_all, "launches": launches, "layout": bp.bp_get_layout(G.h),
           "band_launch_s": band_s / (args.steps * K), "clocks": clk.summary()}

    # end to end through the public API.  Every step starts from host data and
    # reads its MAP back into pinned host memory.  "e2e": the inputs are the
    # stereo pair (two 8-bit images in pinned host memory), handed to the C
    # ABI as host buffers; bp_set_unary_stereo copies them to the device and
    # forms the unary there.  "e2e_unary_upload": the precomputed FP32 unary
    # [H][W][M] is uploaded instead, the next step's upload overlapping the
    # current step on a copy stream (two device staging buffers), and given
    # to bp_set_unary.
    def run_e2e(kind):
        n_e = max(1, args.steps)
        map_host = [torch.empty((cfg.H, cfg.W), dtype=torch.int32).pin_memory() for _ in range(2)]
        if kind == "stereo":
            srcs = [torch.from_numpy(st.left).pin_memory(), torch.from_numpy(st.right).pin_memory()]
            table = wl.unary_table_f32(cfg)
        else:
            srcs = [g_host]
            bufs = [torch.empty_like(g_host, device="cuda") for _ in range(2)]
            copy_stream = torch.cuda.Stream()
            ready = [torch.cuda.Event() for _ in range(2)]
            consumed = [None, None]
        torch.cuda.synchronize()
        clk_e = ClockSampler(dev).__enter__().wait_ready()
        e0 = time.perf_counter()

        def upload(i):
            b = i % 2
            with torch.cuda.stream(copy_stream):
                if consumed[b] is not None:
                    copy_stream.wait_event(consumed[b])
                bufs[b].copy_(g_host, non_blocking=True)
                ready[b].record(copy_stream)
        if kind != "stereo":
            upload(0)
        for i in range(n_e):
            b = i % 2
            if kind == "stereo":
                G.set_unary_stereo(srcs[0], srcs[1], table, cfg.Tu)
            else:
                stream.wait_event(ready[b])
                G.set_unary(bufs[b])
                consumed[b] = torch.cuda.Event()
                consumed[b].record(stream)
                if i + 1 < n_e:
                    upload(i + 1)
            step()
            with torch.cuda.stream(stream):
                map_host[b].copy_(mp, non_blocking=True)
        stream.synchronize()
        G.sync()
        torch.cuda.synchronize()
        e_wall = time.perf_counter() - e0
        clk_e.__exit__()
        return {"value": units_step * n_e * world / e_wall, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(t.numel() * t.element_size() for t in srcs)),
                "d2h_bytes_per_step": int(map_host[0].numel() * 4), "steps": n_e,
                "inputs": ("stereo pair [H][W] uint8 x 2 from pinned host memory through the C ABI; "
                           "unary formed on the device" if kind == "stereo"
                           else "unary [H][W][M] float32 uploaded from pinned host memory"),
                "clocks": clk_e.summary()}

    if not args.no_e2e:
        out["e2e"] = run_e2e("stereo")
        out["e2e_unary_upload"] = run_e2e("unary")
        G.set_unary(g_dev)
        torch.cuda.synchronize()

    # O(M^2) baselines on the same grid and state, timed per iteration: each
    # update (the O(mM) one included, so the ratio is taken under the same
    # conditions) runs `reps` repetitions of `n_it` iterations after a warm-up
    # call; the median repetition is reported, with the clocks of the region.
    if not args.no_baselines:
        out["baselines"] = time_updates_median(
            G, stream, cfg, dev,
            [("band_mM", None), ("dense_bf16_tcgen05_fused", bp.BP_DENSE_BF16_TC_FUSED),
             ("dense_bf16_tcgen05", bp.BP_DENSE_BF16_TC), ("dense_fp32_cuda_core", bp.BP_DENSE_CUDA_CORE)])
    G.close()
    return out


# ------------------------------------------------- secondary workloads ----------
# Each prints its own JSON line; the default run (no --workload) is the line
# above.  They measure the other rows of the hot path on their own workloads.

def _event_time(stream, fn, reps=1):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


def measure_batch(args, n=64, K=30):
    """64 MRFs of uneven size / labels / band, K iterations per step, one
    persistent launch per step; min-sum int32 and sum-product FP32.  Returns
    (per-mode results, workload description)."""
    import torch
    from paper_1010_0012_gb300 import bp
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    items = wl.make_batch(n=n)
    units = sum(wl.directed_edges(it.cfg.W, it.cfg.H) * it.cfg.M for it in items) * K
    bytes_it = sum((it.cfg.W * it.cfg.H * it.cfg.M + 2 * wl.directed_edges(it.cfg.W, it.cfg.H) * it.cfg.M) * 4
                   for it in items)
    stream = torch.cuda.Stream()
    res = {}
    pk = peaks()
    for mode_name, dtype, mode in (("min_i32", bp.BP_I32, bp.BP_MAX), ("sum_f32", bp.BP_F32, bp.BP_SUM)):
        descs, keep = [], []
        for it in items:
            if dtype == bp.BP_F32:
                un = torch.from_numpy(wl.unary_f32(it.stereo)).cuda()
                tab, fb = wl.pair_table_f32(it.cfg.alpha, it.cfg.T)
            else:
                un = torch.from_numpy(wl.unary_i32(it.stereo)).cuda()
                tab, fb = wl.pair_table_i32(it.cfg.alpha, it.cfg.T)
            keep.append(un)
            descs.append((un, tab, it.cfg.T, fb))
        torch.cuda.synchronize()
        b = bp.bp_batch_create(descs, dtype, stream=stream)
        del keep
        tune_ms = bp.bp_batch_autotune(b, mode, 8)
        tiling = {"dominant_class": bp.bp_batch_get_tiling(b),
                  "per_class (Mp, T, family, tile_words)": [bp.bp_batch_get_class_tiling(b, k)
                                                            for k in range(bp.bp_batch_class_count(b))]}

        def step():
            bp.bp_batch_reset_messages(b)
            bp.bp_batch_iterate(b, 0, mode)
            bp.bp_batch_iterate(b, K, mode)
        for _ in range(args.warmup):
            step()
        bp.bp_batch_sync(b)
        l0 = bp.bp_batch_launch_count(b)
        with ClockSampler(dev) as clk:
            clk.wait_ready()
            t = _event_time(stream, step, args.steps)
        bp.bp_batch_sync(b)
        launches = bp.bp_batch_launch_count(b) - l0
        ach = bytes_it * K / t / 1e9
        res[mode_name] = {"value": units / t, "unit": UNIT, "ms_per_step": t * 1e3, "tiling": tiling,
                          "autotune_ms_per_iter": tune_ms, "gpu_launches": launches,
                          "roofline": {"bound": "hbm", "kernel": "batch_kernel (persistent, all MRFs)",
                                       "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                       "frac": ach / pk["hbm_gbs"], "peak_source": pk["source"],
                                       "algorithmic_bytes_per_iteration": bytes_it},
                          "clocks": clk.summary()}
        bp.bp_batch_destroy(b)
        torch.cuda.empty_cache()
    desc = (f"batch of {n} MRFs, W 128..640, H 128..480, M in 32/64/128/256, T 2..8, {K} synchronous iterations "
            "per step, one persistent launch")
    return res, {"workload": desc, "algorithmic_bytes_per_iteration": bytes_it, "units_per_step": units}


def run_batch_workload(args):
    n = 64 if not args.rows else max(2, args.rows)
    res, config = measure_batch(args, n=n)
    line = {"metric": METRIC + " (batch of uneven MRFs)", "value": res["min_i32"]["value"], "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["min_i32"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i32", "data": "synthetic", "config": config, "modes": res}
    print(json.dumps(line))


def measure_dense_compare(args, pairs=((64, 3), (128, 4), (256, 4)), cuda_core=True, reps=5):
    """The O(mM) update against the O(M^2) baselines on the same 1280x720
    grid at each (M, T): time per synchronous sum-product iteration of each
    (CUDA events on the handle's stream, median of `reps` runs after a
    warm-up run), with the sampled clocks of the region."""
    import dataclasses
    import torch
    from paper_1010_0012_gb300 import bp
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    pk = peaks()
    out = {}
    for M, T in pairs:
        cfg = dataclasses.replace(wl.CONFIGS["grid1280x720_m128"], M=M, T=T)
        st = wl.make_stereo(cfg)
        u = torch.from_numpy(wl.unary_f32(st)).cuda()
        torch.cuda.synchronize()
        G = bp.BPGrid(cfg.W, cfg.H, M, bp.BP_F32, stream=stream)
        G.set_unary(u)
        tab, fbar = wl.pair_table_f32(cfg.alpha, T)
        G.set_potential(tab, T, fbar)
        kinds = [("band_mM", None, 5), ("dense_bf16_tcgen05_fused", bp.BP_DENSE_BF16_TC_FUSED, 5),
                 ("dense_bf16_tcgen05", bp.BP_DENSE_BF16_TC, 5)]
        if cuda_core:
            kinds.append(("dense_fp32_cuda_core", bp.BP_DENSE_CUDA_CORE, 1 if M > 128 else 5))
        res = {}
        with ClockSampler(dev) as clk:
            clk.wait_ready()
            for name, kind, n_it in kinds:
                if kind is None:
                    fn = (lambda n: (lambda: G.iterate(n, bp.BP_SUM, "sync")))(n_it)
                else:
                    fn = (lambda k, n: (lambda: bp.bp_iterate_dense(G.h, n, k)))(kind, n_it)
                try:
                    G.reset()
                    G.iterate(0, bp.BP_SUM, "sync")
                    fn()
                    G.sync()
                    ts = []
                    for _ in range(reps):
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        fn()
                        b.record(stream)
                        b.synchronize()
                        ts.append(a.elapsed_time(b) / 1e3 / n_it)
                    G.sync()
                except bp.BPError as e:
                    res[name] = {"unavailable": str(e)[:160]}
                    continue
                t = statistics.median(ts)
                ach = workload_units(cfg) * UPDATE_BYTES[name] / t / 1e9
                res[name] = {"value": workload_units(cfg) / t, "unit": UNIT, "ms_per_iter": t * 1e3,
                             "ms_per_iter_min_max": [min(ts) * 1e3, max(ts) * 1e3],
                             "roofline": {"bound": "hbm", "bytes_per_update": UPDATE_BYTES[name], "achieved": ach,
                                          "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                                          "peak_source": pk["source"]}}
        res["clocks"] = clk.summary()
        if "value" in res.get("band_mM", {}) and "value" in res.get("dense_bf16_tcgen05_fused", {}):
            res["band_over_fused_tcgen05"] = res["band_mM"]["value"] / res["dense_bf16_tcgen05_fused"]["value"]
        res["layout"] = list(bp.bp_get_layout(G.h))
        out[f"M{M}_T{T}"] = res
        G.close()
        del u
        torch.cuda.empty_cache()
    return out


def run_dense_compare_workload(args):
    out = measure_dense_compare(args)
    first = next(iter(out.values()))
    line = {"metric": METRIC + " vs the O(M^2) baselines", "value": first["band_mM"]["value"], "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "1280x720 random-dot stereo, synchronous sum-product, M = 64 (T = 3), "
                                   "M = 128 (T = 4) and M = 256 (T = 4); the O(M^2) updates run on the same grid "
                                   "and state"},
            "peak_source": peaks()["source"], "modes": out}
    print(json.dumps(line))


def l2_copy_probe(stream, mb=16, reps=200):
    """A like-for-like bandwidth for workloads whose working set stays in L2:
    a device-to-device copy between two `mb` MB buffers (both fit in L2 with
    room to spare), repeated `reps` times after a warm-up, timed with CUDA
    events; read plus write bytes per second.  At 16 MB a copy moves 32 MB
    per launch, what one red-black half-step of 384x288, M = 16 moves, so it
    carries the same per-launch ramp and tail; it is not the L2 peak."""
    import torch
    n = mb * (1 << 20) // 4
    with torch.cuda.stream(stream):
        a = torch.ones(n, dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        for _ in range(10):
            b.copy_(a)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            b.copy_(a)
        e1.record(stream)
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    return {"copy_gbs": 2 * n * 4 / t / 1e9,
            "how": f"copy between two {mb} MB device buffers ({2 * mb} MB per launch), {reps} repetitions, "
                   "CUDA events"}


def measure_grid(args, name):
    """A single grid in both modes on its own schedule (e.g. 384x288 red-black).
    Returns (per-mode results, workload description)."""
    import torch
    from paper_1010_0012_gb300 import bp
    cfg = wl.CONFIGS[name]
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    st = wl.make_stereo(cfg)
    stream = torch.cuda.Stream()
    pk = peaks()
    units = workload_units(cfg) * cfg.iters
    res = {}
    for mode_name, dtype, mode, un, tabfb in (
            ("sum_f32", bp.BP_F32, bp.BP_SUM, wl.unary_f32(st), wl.pair_table_f32(cfg.alpha, cfg.T)),
            ("min_i32", bp.BP_I32, bp.BP_MAX, wl.unary_i32(st), wl.pair_table_i32(cfg.alpha, cfg.T))):
        if mode_name.split("_")[0] not in cfg.modes:
            continue
        u = torch.from_numpy(un).cuda()
        torch.cuda.synchronize()
        G = bp.BPGrid(cfg.W, cfg.H, cfg.M, dtype, stream=stream)
        bp.bp_set_persistent(G.h, args.persistent)
        G.set_unary(u)
        G.set_potential(tabfb[0], cfg.T, tabfb[1])

        def step():
            G.reset()
            G.iterate(0, mode, cfg.schedule)
            G.iterate(cfg.iters, mode, cfg.schedule)
        for _ in range(args.warmup):
            step()
        G.sync()
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            clk.wait_ready()
            t = _event_time(stream, step, args.steps)
        G.sync()
        ach = algorithmic_bytes(cfg) * cfg.iters / t / 1e9
        res[mode_name] = {"value": units / t, "unit": UNIT, "ms_per_step": t * 1e3,
                          "layout": list(bp.bp_get_layout(G.h)),
                          "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                       "frac": ach / pk["hbm_gbs"], "peak_source": pk["source"],
                                       "note": "working set fits in L2 when small: frac may exceed 1"},
                          "clocks": clk.summary()}
        G.close()
    state_bytes = (cfg.W * cfg.H * cfg.M * 4) * (9 if cfg.schedule == "sync" else 5)
    if state_bytes < 64 << 20:
        # the working set stays in the 129 MB L2: report against a measured
        # L2 copy bandwidth as well as against HBM
        probe = l2_copy_probe(stream)
        for r in res.values():
            r["roofline"]["l2_probe"] = dict(probe, frac=r["roofline"]["achieved"] / probe["copy_gbs"])
    desc = f"{cfg.name}: {cfg.W}x{cfg.H}, M={cfg.M}, T={cfg.T}, {cfg.iters} {cfg.schedule} iterations per step"
    return res, {"workload": desc}


def run_grid_workload(args, name):
    res, config = measure_grid(args, name)
    first = next(iter(res.values()))
    line = {"metric": METRIC, "value": first["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": first["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config, "modes": res}
    print(json.dumps(line))


def gradient_floor_bytes(cfg, every=5):
    """HBM bytes the checkpointed gradient's launches must move: the recorded
    forward (K log-domain iterations at 9 bytes per update, its checkpoints
    written in place), one copy of the starting state into the first
    checkpoint, the recomputed states of every segment but the last (whose
    states the forward keeps), and K adjoint launches at 15 bytes per
    node-label-direction (read l, log g, the adjoint in and d log g; write the
    adjoint out and d log g).  Beliefs, their reverse and the 8-byte scale per
    message are left out (under 2 %)."""
    nodes = cfg.W * cfg.H
    De = wl.directed_edges(cfg.W, cfg.H)
    K = cfg.iters
    n_ck = (K + every - 1) // every
    last_len = K - (n_ck - 1) * every
    fwd = (nodes * cfg.M + 2 * De * cfg.M) * 4
    adj = nodes * cfg.M * 15 * 4
    state = 4 * nodes * cfg.M * 4
    parts = {"forward": K * fwd, "checkpoints": 2 * state, "recompute": (K - n_ck - (last_len - 1)) * fwd,
             "adjoint": K * adj}
    return sum(parts.values()), parts


def measure_gradient(args, every=5):
    """Loss and gradient (alpha, fbar, beta) of 30 unrolled log-domain
    iterations on 256x256, M=64, T=3, checkpoint every 5.  Wall-clock time per
    gradient (the call a user makes: forward, loss, backward, the three
    gradients read back to the host), against the byte floor of its launches."""
    import torch
    from paper_1010_0012_gb300 import autograd, bp
    cfg = wl.CONFIGS["grid256_m64_grad"]
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    st = wl.make_stereo(cfg)
    cost = torch.from_numpy(st.cost.astype(np.float32)).cuda()
    gt = torch.as_tensor(st.d_gt, dtype=torch.long).cuda()
    # the handle orders its work on torch's stream: no host synchronisation
    # between the library's kernels and torch's
    G = bp.BPGrid(cfg.W, cfg.H, cfg.M, bp.BP_F32, stream=torch.cuda.current_stream())
    # the parameters live on the GPU, as in a training loop: the reverse pass
    # keeps their gradients on the device and the step waits once, when the
    # three gradients are read back
    a = torch.tensor(cfg.alpha, device="cuda", requires_grad=True)
    fb = torch.tensor(float(np.exp(-cfg.alpha * cfg.T)), device="cuda", requires_grad=True)
    be = torch.tensor(cfg.beta, device="cuda", requires_grad=True)

    def step():
        a.grad = fb.grad = be.grad = None
        loss = autograd.stereo_nll(cost, gt, a, fb, be, cfg.T, cfg.iters, G, every)
        loss.backward()
        return torch.stack([a.grad, fb.grad, be.grad]).cpu()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = G.launches
    with ClockSampler(dev) as clk:
        clk.wait_ready()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        t = (time.perf_counter() - t0) / args.steps
    launches = G.launches - l0
    G.close()
    pk = peaks()
    floor, parts = gradient_floor_bytes(cfg, every)
    ach = floor / t / 1e9
    return {"value": 1.0 / t, "unit": "gradients/s", "ms_per_gradient": t * 1e3,
            "forward_message_updates_per_s": workload_units(cfg) * cfg.iters / t,
            "gpu_launches_per_gradient": launches / max(1, args.steps),
            "roofline": {"bound": "hbm", "kernel": "whole gradient (log forward, checkpoints, recompute, adjoint)",
                         "algorithmic_bytes_per_gradient": floor, "bytes_by_part": parts,
                         "floor_ms": floor / (pk["hbm_gbs"] * 1e9) * 1e3, "achieved": ach, "peak": pk["hbm_gbs"],
                         "unit": "GB/s", "frac": ach / pk["hbm_gbs"], "peak_source": pk["source"]},
            "clocks": clk.summary(), "timing": f"wall clock over {args.steps} gradients after {args.warmup}"}, {
        "workload": "256x256, M=64, T=3, 30 log-domain iterations, checkpoint 5, loss -sum log b(gt); "
                    "gradients wrt alpha, fbar, beta"}


def run_gradient_workload(args):
    res, config = measure_gradient(args)
    line = {"metric": "gradient evaluations/s (forward + adjoint, 30 unrolled iterations)", "value": res["value"],
            "unit": "gradients/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["ms_per_gradient"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config, "result": res}
    print(json.dumps(line))


def run_multiscale_workload(args):
    """Time to a disparity map: single-scale iterations against coarse-to-fine
    schedules on the 1280x720, M=128 workload (sum-product, synchronous), with
    the share of pixels whose MAP is more than one disparity off the truth."""
    import torch
    from paper_1010_0012_gb300 import bp
    cfg = wl.CONFIGS["grid1280x720_m128"]
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    st = wl.make_stereo(cfg)
    stream = torch.cuda.Stream()
    u = torch.from_numpy(wl.unary_f32(st)).cuda()
    torch.cuda.synchronize()
    G = bp.BPGrid(cfg.W, cfg.H, cfg.M, bp.BP_F32, stream=stream)
    G.set_unary(u)
    tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
    G.set_potential(tab, cfg.T, fbar)
    gt = torch.from_numpy(st.d_gt).cuda()
    runs = {}
    plans = [("single", [k]) for k in (10, 30, 100)] + \
            [("multiscale", p) for p in ([10, 10, 10, 10, 10], [20, 10, 5, 5, 5, 5], [30, 20, 10, 5])]
    for kind, plan in plans:
        def step():
            G.reset()
            if kind == "single":
                G.iterate(plan[0], bp.BP_SUM, "sync")
            else:
                bp.bp_iterate_multiscale(G.h, plan, bp.BP_SUM, bp.BP_SYNC)
        for _ in range(args.warmup):
            step()
        G.sync()
        t = _event_time(stream, step, args.steps)
        _, mp = G.beliefs()
        G.sync()
        torch.cuda.synchronize()
        err = float(((mp - gt).abs() > 1).float().mean())
        runs[f"{kind}:{'-'.join(map(str, plan))}"] = {"ms": t * 1e3, "map_error_gt1": err,
                                                       "fine_iterations": plan[-1]}
    line = {"metric": "time to disparity map (ms) and MAP error, single-scale vs coarse-to-fine",
            "value": runs["multiscale:10-10-10-10-10"]["ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "1280x720, M=128, T=4, sum-product, synchronous; levels coarsest first"},
            "runs": runs}
    G.close()
    print(json.dumps(line))


def measure_sparse(args):
    """The O(nnz) kernel on the 1280x720, M=128 grid with a potential that is
    not a function of x_i - x_j: 9 compatible sender labels per receiver label
    drawn at random (seed 7) with random values; message updates/s of the
    register-pattern and the list kernels, sum-product and min-sum."""
    import torch
    from paper_1010_0012_gb300 import bp
    cfg = wl.CONFIGS["grid1280x720_m128"]
    if args.rows:
        import dataclasses
        cfg = dataclasses.replace(cfg, H=min(args.rows, cfg.H))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    st = wl.make_stereo(cfg)
    rng = np.random.default_rng(7)
    rowptr, cols, vals = [0], [], []
    for xj in range(cfg.M):
        xs = rng.choice(cfg.M, size=9, replace=False)
        cols.extend(int(x) for x in xs)
        vals.extend(float(v) for v in rng.uniform(0.2, 1.0, 9))
        rowptr.append(len(cols))
    stream = torch.cuda.Stream()
    res = {}
    pk = peaks()
    units = workload_units(cfg) * 10
    for name, dtype, mode, un in (("sum_f32", bp.BP_F32, bp.BP_SUM, wl.unary_f32(st)),
                                  ("min_i32", bp.BP_I32, bp.BP_MAX, wl.unary_i32(st))):
        u = torch.from_numpy(un).cuda()
        torch.cuda.synchronize()
        G = bp.BPGrid(cfg.W, cfg.H, cfg.M, dtype, stream=stream)
        G.set_unary(u)
        if dtype == bp.BP_F32:
            bp.bp_set_potential_sparse(G.h, rowptr, cols, vals, 0.1, dtype)
        else:
            bp.bp_set_potential_sparse(G.h, rowptr, cols, [int(10 * v) for v in vals], 10, dtype)

        def step():
            G.reset()
            G.iterate(0, mode)
            G.iterate(10, mode)
        res[name] = {}
        for kname, kind in (("registers", bp.BP_SPARSE_REGISTERS), ("lists", bp.BP_SPARSE_LISTS)):
            try:
                bp.bp_set_sparse_kernel(G.h, kind)
            except bp.BPError as e:
                res[name][kname] = {"unavailable": str(e)[:160]}
                continue
            _, steps_, wf = bp.bp_get_sparse_kernel(G.h)
            for _ in range(args.warmup):
                step()
            G.sync()
            with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
                clk.wait_ready()
                t = _event_time(stream, step, args.steps)
            G.sync()
            ach = algorithmic_bytes(cfg) * 10 / t / 1e9
            res[name][kname] = {"value": units / t, "unit": UNIT, "ms_per_iter": t * 1e2,
                                "schedule": {"steps": steps_, "gather_wavefronts_per_node": wf},
                                "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"],
                                             "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                                             "peak_source": pk["source"]},
                                "clocks": clk.summary()}
        G.close()
        del u
    return res, {"workload": f"{cfg.W}x{cfg.H}, M={cfg.M}, random non-difference pattern (9 sender labels per "
                             "receiver label, seed 7), 10 synchronous iterations per step; no L2 flush: each "
                             "iteration streams 4.2 GB"}


def run_sparse_workload(args):
    res, config = measure_sparse(args)
    line = {"metric": METRIC + " (general sparse compatibility, 9 pairs per label)",
            "value": res["sum_f32"]["registers"].get("value", res["sum_f32"]["lists"].get("value")), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": config, "modes": res}
    print(json.dumps(line))


def measure_factor(args, with_dense=True):
    """Sec. 7's three-variable factors: a second-order smoothness model on a
    256x256 stereo grid with M=32 labels.  Every horizontal and vertical run of
    three pixels is a factor with f = exp(-alpha |x0 - 2 x1 + x2|) where the
    second difference is at most 1 (C = compatible triplets) and fbar =
    exp(-2 alpha) elsewhere.  Factor-to-variable message entries per second of
    the O(C + M) update, and (with_dense) of the standard O(M^3) update."""
    import torch
    from paper_1010_0012_gb300 import bp
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfg = wl.small_config("fg256", 256, 256, 32, 1, alpha=1.0, structure="planar", seed=1006)
    st = wl.make_stereo(cfg)
    W, H, M, alpha = cfg.W, cfg.H, cfg.M, 1.0
    idx = np.arange(W * H).reshape(H, W)
    fs = np.concatenate([np.stack([idx[:, :-2].ravel(), idx[:, 1:-1].ravel(), idx[:, 2:].ravel()], 1),
                         np.stack([idx[:-2].ravel(), idx[1:-1].ravel(), idx[2:].ravel()], 1)]).astype(np.int32)
    x0, x1, x2 = np.meshgrid(np.arange(M), np.arange(M), np.arange(M), indexing="ij")
    d2 = np.abs(x0 - 2 * x1 + x2)
    keep = d2 <= 1
    trip = np.stack([x0[keep], x1[keep], x2[keep]], 1).astype(np.int32)
    vals = np.exp(-alpha * d2[keep].astype(np.float64)).astype(np.float32)
    fbar = float(np.float32(np.exp(-2 * alpha)))
    g = torch.from_numpy(wl.unary_f32(st).reshape(W * H, M)).cuda()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    G = bp.bp_fg_create(W * H, M, fs, bp.BP_F32, stream=stream)
    bp.bp_fg_set_unary(G, g)
    bp.bp_fg_set_factor(G, trip, vals, fbar, bp.BP_F32)
    units = len(fs) * 3 * M
    res = {}
    modes = (("sparse_O(C+M)", bp.bp_fg_iterate, 10),) + \
        ((("dense_O(M^3)", bp.bp_fg_iterate_dense, 2),) if with_dense else ())
    for name, fn, K in modes:
        def step():
            bp.bp_fg_reset_messages(G)
            fn(G, K, bp.BP_SUM)
        for _ in range(max(1, args.warmup)):
            step()
        bp.bp_fg_sync(G)
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            clk.wait_ready()
            t = _event_time(stream, step, args.steps)
        bp.bp_fg_sync(G)
        res[name] = {"value": units * K / t, "unit": "factor-to-variable message entries/s",
                     "ms_per_iter": t * 1e3 / K, "clocks": clk.summary()}
    bp.bp_fg_destroy(G)
    # roofline of the O(C + M) iteration: every triplet contributes one term to
    # each of the three messages of every factor (n_factors * 3 * C terms per
    # iteration); per 32 terms a warp spends four L1 / shared-memory data-pipe
    # wavefronts (two 4-byte gathers of the incoming messages and the 8-byte
    # entry read through L1), one wavefront per cycle per SM
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", 2070.0)) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 2070.0
    terms = len(fs) * 3 * len(trip)
    t_it = res["sparse_O(C+M)"]["ms_per_iter"] / 1e3
    peak_terms = props.multi_processor_count * sm_mhz * 1e6 * 32 / 4
    res["sparse_O(C+M)"]["roofline"] = {
        "bound": "alu", "resource": "L1 / shared-memory data pipe: 4 wavefronts per 32 triplet terms",
        "achieved": terms / t_it / 1e9, "peak": peak_terms / 1e9, "unit": "G terms/s",
        "frac": terms / t_it / peak_terms, "terms_per_iteration": terms,
        "hbm_bytes_per_iteration": len(fs) * 6 * M * 4 + W * H * M * 4 * 2,
        "hbm_frac": (len(fs) * 6 * M * 4 + W * H * M * 4 * 2) / t_it / (peaks()["hbm_gbs"] * 1e9)}
    if with_dense:
        res["speedup"] = res["sparse_O(C+M)"]["value"] / res["dense_O(M^3)"]["value"]
    return res, {"workload": f"256x256 grid, M={M}, {len(fs)} triplet factors, C={len(trip)} of M^3={M ** 3}, "
                             "10 flooding iterations per step"}


def run_factor_workload(args):
    res, config = measure_factor(args)
    line = {"metric": "factor BP message entries/s, O(C) vs O(M^3) (three-variable factors)",
            "value": res["sparse_O(C+M)"]["value"], "unit": "entries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": config, "modes": {k: v for k, v in res.items() if k != "speedup"}, "speedup": res["speedup"]}
    print(json.dumps(line))


def main():
    args = parse_args()
    if args.impl == "ours" and args.workload == "dense_compare":
        run_dense_compare_workload(args)
        return 0
    if args.impl == "ours" and args.workload == "factor256":
        run_factor_workload(args)
        return 0
    if args.impl == "ours" and args.workload == "multiscale1280x720":
        run_multiscale_workload(args)
        return 0
    if args.impl == "ours" and args.workload == "sparse1280x720":
        run_sparse_workload(args)
        return 0
    if args.impl == "ours" and args.workload == "batch64":
        run_batch_workload(args)
        return 0
    if args.impl == "ours" and args.workload == "grid256_m64_grad":
        run_gradient_workload(args)
        return 0
    if args.impl == "ours" and args.workload in ("grid32_m16", "grid384x288_m16"):
        run_grid_workload(args, args.workload)
        return 0
    cfg = wl.CONFIGS[args.workload]
    if args.rows:
        import dataclasses
        cfg = dataclasses.replace(cfg, H=min(args.rows, cfg.H))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    config = {"workload": f"{cfg.name}: {cfg.W}x{cfg.H} grid, M={cfg.M}, T={cfg.T} (m={2 * cfg.T + 1}), "
                          f"alpha={cfg.alpha}, {cfg.iters} synchronous sum-product iterations + beliefs/MAP "
                          f"per step, random-dot stereo (seed {cfg.seed})",
              "W": cfg.W, "H": cfg.H, "M": cfg.M, "T": cfg.T, "iters_per_step": cfg.iters,
              "l2": "no flush: each iteration streams "
                    f"{algorithmic_bytes(cfg) / 1e9:.2f} GB, far above the 129 MB L2",
              "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}

    if args.impl == "reference":
        if rank != 0:
            return 0
        st = wl.make_stereo(cfg)
        times, units = [], 0
        desc = ""
        for i in range(args.warmup + args.steps):
            v, desc, t = oracle_sample(cfg, st, target_s=2.0)
            if i >= args.warmup:
                times.append(t)
                units += v * t
        tot = sum(times)
        val = units / tot
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": "each step: " + desc},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    res = run_ours(args, cfg, rank, world)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    pk = peaks()
    per_launch_bytes = algorithmic_bytes(cfg)
    achieved = per_launch_bytes / res["band_launch_s"] / 1e9
    value = res["units"] / res["elapsed"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * res["elapsed"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
            "roofline": {"bound": "hbm", "kernel": f"band_sum_kernel<{res['layout'][0]},{res['layout'][1]},{cfg.T}>",
                         "achieved": achieved,
                         "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                         "peak_source": pk["source"], "algorithmic_bytes_per_launch": per_launch_bytes,
                         "traffic": recorded_traffic(f"band_sum_kernel<{res['layout'][0]},{res['layout'][1]},{cfg.T}>",
                                                     cfg)},
            "clocks": res["clocks"], "gpu_launches": res["launches"]}
    if "e2e" in res:
        line["e2e"] = res["e2e"]
        line["e2e_unary_upload"] = res["e2e_unary_upload"]
    if "baselines" in res:
        line["baselines"] = res["baselines"]
    if not args.no_secondary and world == 1:
        # the other workloads of the hot path, each with its own roofline and
        # clocks: the 384x288 red-black grid (both modes), the 64-MRF batch
        # (both modes), the checkpointed gradient, the O(mM) update against
        # the tensor-core O(M^2) update at 256 labels, the general sparse
        # potential (both kernels, both modes) and the three-variable factor
        # graph (the O(C + M) update; its O(M^3) comparison only in its own run)
        sec_args = argparse.Namespace(**vars(args))
        sec_args.steps, sec_args.warmup = max(3, min(args.steps, 10)), max(3, min(args.warmup, 3))
        sec = {}
        for key, fn in (("grid384x288_m16", lambda: measure_grid(sec_args, "grid384x288_m16")),
                        ("batch64", lambda: measure_batch(sec_args)),
                        ("grid256_m64_grad", lambda: measure_gradient(sec_args)),
                        ("dense_compare_m256", lambda: (measure_dense_compare(sec_args, ((256, 4),), cuda_core=False),
                                                        {"workload": "1280x720, M = 256, T = 4, synchronous "
                                                                     "sum-product: O(mM) band against the fused and "
                                                                     "packed BF16 tcgen05 O(M^2) updates"})),
                        ("sparse1280x720", lambda: measure_sparse(sec_args)),
                        ("factor256", lambda: measure_factor(sec_args, with_dense=False))):
            try:
                r, c = fn()
                sec[key] = {"config": c, "steps": sec_args.steps, "warmup": sec_args.warmup, "result": r}
            except Exception as e:      # a failed secondary line must not lose the headline
                sec[key] = {"unavailable": f"{type(e).__name__}: {str(e)[:200]}"}
        line["secondary"] = sec
    if not args.no_cpu_baseline:
        st = wl.make_stereo(cfg)
        v, desc, t = oracle_sample(cfg, st, target_s=10.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
    if not args.no_cpu_throughput:
        line["cpu_throughput"] = cpu_throughput_sample(cfg, wl.make_stereo(cfg))
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
