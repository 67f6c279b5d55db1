#!/usr/bin/env python
"""Benchmark: L.A.Cosmic Mpix/s at niter=4 on a 9576 x 6388 uint16 frame.

Workload: the 61-Mpx uint16 large-format CMOS frame (seed 1; sky 300 ADU,
gain 0.8, rn 1.2, ~4000 stars, 150000 cosmic-ray tracks, 0.5% salt-and-
pepper), sigclip 4.5, sigfrac 0.3, objlim 5, niter 4, one frame per call.
A step is one full detect-and-clean of the frame (all iterations plus the
final mask/cleaned write).  Inputs are resident in HBM when timing starts;
L2 is flushed (a 256 MiB write) between timed steps.  With --gpus N (under
torchrun) every rank cleans its own frame: weak scaling, no collective.

--impl reference times the float32 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "lacosmic_9576x6388_u16_niter4"

# DRAM bytes (read + write) per core_kernel launch from one ncu capture on
# this workload, keyed by kernel_source_sha() of the captured build; any other
# source reports null (the counters no longer describe the kernel).
NCU_CORE_TRAFFIC = {"f6175d2fa2a59759": 149_255_936}


def kernel_source_sha() -> str:
    """sha256 prefix of the device code: the kernel sources with // comments
    and blank lines dropped, so a comment edit keeps the recorded counters."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in ("lacos_kernels.cuh", "networks.cuh", "gain_math.cuh", "lacos.cu"):
        with open(os.path.join(ROOT, "paper_2602_17938_gb300", "csrc", name)) as f:
            for line in f:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


METRIC = "L.A.Cosmic Mpix/s at niter=4 on 61-Mpx frames"
E2E_DEPTH = 3  # host-to-host requests in flight in the e2e measurement


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=5)
    return ap.parse_args()


def dist_env():
    from paper_2602_17938_gb300 import dist as pdist
    return pdist.env()


# ---------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(self.out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax.append(float(row[2]))
            except ValueError:
                continue
            for nm, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- CPU oracle ----
def oracle_sample(frame, spec, seconds_target=12.0, crop=256):
    """Time the float32 CPU oracle on crops of the frame (one core)."""
    import numpy as np
    import oracle
    oracle.build()
    ny, nx = frame.shape
    rng = np.random.default_rng(123)
    done_px, t_total, n = 0, 0.0, 0
    while t_total < seconds_target and n < 64:
        y0 = int(rng.integers(0, ny - crop))
        x0 = int(rng.integers(0, nx - crop))
        c = np.ascontiguousarray(frame[y0:y0 + crop, x0:x0 + crop])
        t0 = time.perf_counter()
        oracle.run(c, spec.gain, spec.readnoise, spec.satlevel, spec.sigclip, spec.sigfrac,
                   spec.objlim, spec.niter)
        t_total += time.perf_counter() - t0
        done_px += crop * crop
        n += 1
    return {"value": done_px / 1e6 / t_total, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} crops of {crop}x{crop} px from the workload frame, niter=4, "
                      f"single-threaded float32 C++ oracle, {t_total:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2602_17938_gb300 import synth
    spec = synth.config_specs(1)[0]
    frame = synth.make_frame(spec)
    import numpy as np
    import oracle
    oracle.build()
    crop = 192
    rng = np.random.default_rng(7)
    ny, nx = frame.shape

    def step():
        y0, x0 = int(rng.integers(0, ny - crop)), int(rng.integers(0, nx - crop))
        c = np.ascontiguousarray(frame[y0:y0 + crop, x0:x0 + crop])
        oracle.run(c, spec.gain, spec.readnoise, spec.satlevel, spec.sigclip, spec.sigfrac,
                   spec.objlim, spec.niter)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = args.steps * crop * crop / 1e6 / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{crop}x{crop} crop per step",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": f"one {crop}x{crop} crop of the workload frame per step, "
                                       "niter=4, single-threaded float32 C++ oracle"},
            "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ batched and served ---
def run_batched(args, dev):
    """64 frames of uneven sizes (2048^2 f32, 4096x3072 u16, 9576x6388 u16; the
    config-1 recipe with per-frame gain and read noise) in one request: one
    launch per iteration level over a shared tile queue, replayed as a CUDA graph."""
    import torch
    from paper_2602_17938_gb300 import lacos, synth
    specs = synth.config_specs(2)
    t0 = time.perf_counter()
    frames = synth.make_frames_parallel(specs)
    gen_s = time.perf_counter() - t0
    d_frames = [lacos.to_device(f, dev) for f in frames]
    del frames
    masks = [torch.empty(f.shape, dtype=torch.uint8, device=dev) for f in d_frames]
    cleans = [torch.empty(f.shape, dtype=torch.float32, device=dev) for f in d_frames]
    params = [lacos.make_params(sp.gain, sp.readnoise, sp.satlevel, sp.sigclip, sp.sigfrac,
                                sp.objlim, sp.niter) for sp in specs]
    npix = sum(sp.npix for sp in specs)
    ctx = lacos.Context(dev.index or 0, hbm_budget_bytes=96 << 30, max_slots=2)
    stream = torch.cuda.current_stream(dev)
    t, _ = ctx.submit_batch(d_frames, params, masks, cleans, reuse_graph=True)  # capture
    ctx.wait(t)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.batched_steps)]
    flagged = 0
    for a, b in ev:
        a.record(stream)
        t, per = ctx.submit_batch(d_frames, params, masks, cleans, reuse_graph=True)
        b.record(stream)
        r = ctx.wait(t)
        flagged = r.n_flagged
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    ctx.close()
    del d_frames, masks, cleans
    torch.cuda.empty_cache()
    return {"workload": "64 frames: 16x 2048x2048 f32, 16x 4096x3072 u16, 32x 9576x6388 u16 "
                        "(seed 2), niter=4, one request, CUDA-graph replay",
            "mpix_per_s": npix / 1e6 / (sum(ms) / 1e3 / len(ms)), "ms_per_batch": sum(ms) / len(ms),
            "mpix_per_batch": npix / 1e6, "steps": len(ms), "n_flagged": flagged,
            "frame_generation_s": gen_s, "l2": "inputs (4.6 GB) far exceed L2"}


def run_serving(args, dev):
    """Poisson stream of 9576x6388 u16 frames with 10% 2048x2048 f32 frames,
    admitted by a 120 GB HBM budget, requests overlapping on the device."""
    import math
    import torch
    from paper_2602_17938_gb300 import lacos, serve, synth
    specs = synth.config_specs(3, count=200)
    big = [sp for sp in specs if sp.ny == 6388][:4]
    small = [sp for sp in specs if sp.ny == 2048][:2]
    pool_specs = big + small
    pool = [lacos.to_device(f, dev) for f in synth.make_frames_parallel(pool_specs)]
    p = lacos.make_params(1.0, 1.5)
    kinds = [0 if sp.ny == 6388 else 1 for sp in specs]
    points = []
    with serve.Server(dev.index or 0, hbm_budget_bytes=120 << 30, max_slots=96) as srv:
        # Warm-up: every slot the sweep can use gets its stream and scratch.
        srv.run([serve.Request(pool[i % 4], p, 0.0) for i in range(96)])
        for rate, n in ((1.1, 12), (8.0, 48), (32.0, 120), (math.inf, 160)):
            arr = synth.poisson_arrivals(rate, n) if math.isfinite(rate) else [0.0] * n
            reqs = []
            for i in range(n):
                fr = pool[i % 4] if kinds[i % len(kinds)] == 0 else pool[4 + i % 2]
                reqs.append(serve.Request(fr, p, float(arr[i] - arr[0])))
            st = srv.run(reqs)
            points.append({"rate_hz": rate if math.isfinite(rate) else "saturation", "requests": n,
                           "p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "mean_ms": st.mean_ms,
                           "mpix_per_s": st.mpix_per_s, "max_in_flight": st.max_in_flight})
    del pool
    torch.cuda.empty_cache()
    return {"workload": "Poisson arrivals of 9576x6388 u16 frames, 10% 2048x2048 f32 (seed 3); "
                        "6 distinct frames reused round-robin; 120 GB HBM budget; lacos_submit_async",
            "points": points}


# ------------------------------------------------------------- GPU arm -----
def alu_peak():
    import ctypes
    from paper_2602_17938_gb300 import build
    lib = ctypes.CDLL(build.PEAK_LIB)
    lib.alu_minmax_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]
    f32, u16 = ctypes.c_double(), ctypes.c_double()
    if lib.alu_minmax_peak(0, ctypes.byref(f32), ctypes.byref(u16)) != 0:
        return None, None
    return f32.value, u16.value


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_17938_gb300 import lacos, synth, netcost

    from paper_2602_17938_gb300 import dist as pdist
    spec = synth.config_specs(1)[0]
    spec.seed = pdist.frame_seed(1, rank)
    frame = synth.make_frame(spec)
    ny, nx = frame.shape
    npix = ny * nx
    d_frame = lacos.to_device(frame, dev)
    d_mask = torch.empty((ny, nx), dtype=torch.uint8, device=dev)
    d_clean = torch.empty((ny, nx), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    params = lacos.make_params(spec.gain, spec.readnoise, spec.satlevel, spec.sigclip,
                               spec.sigfrac, spec.objlim, spec.niter)
    ctx = lacos.Context(local)
    stream = torch.cuda.current_stream(dev)
    from paper_2602_17938_gb300 import autotune
    variant, variant_ms = autotune.tune(ctx, d_frame, params, d_mask, d_clean)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        flush.zero_()
        ctx.wait(ctx.submit(d_frame, params, d_mask, d_clean))
    torch.cuda.synchronize()

    ctx.set_profiling(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        profs = []
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            t = ctx.submit(d_frame, params, d_mask, d_clean)
            ev[i][1].record(stream)
            ctx.wait(t)
            profs.append(ctx.last_profile())
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    barrier()
    ctx.set_profiling(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]

    # Optional modes on the same frame, timed the same way (device, L2 flushed).
    modes = {}
    for name, extra in (("default", dict()), ("satgrow2", dict(satgrow=2)), ("sepmed", dict(sepmed=True)),
                        ("gain_estimated", dict(gain=0.0))):
        kw = dict(gain=spec.gain, readnoise=spec.readnoise, satlevel=spec.satlevel, sigclip=spec.sigclip,
                  sigfrac=spec.sigfrac, objlim=spec.objlim, niter=spec.niter, fine_norm=True)
        kw.update(extra)
        mp = lacos.make_params(**kw)
        for _ in range(2):
            ctx.wait(ctx.submit(d_frame, mp, d_mask, d_clean))
        mev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for e0, e1 in mev:
            flush.zero_()
            e0.record(stream)
            t = ctx.submit(d_frame, mp, d_mask, d_clean)
            e1.record(stream)
            ctx.wait(t)
        ms = sum(e0.elapsed_time(e1) for e0, e1 in mev) / len(mev)
        modes[name] = {"params": extra, "ms_per_step": ms, "mpix_per_s": npix / ms / 1e3}
    total_s = pdist.max_over_ranks(sum(step_ms) / 1e3, dev)
    value = pdist.job_throughput(npix, args.steps, ws, total_s)

    # Roofline of the dominant kernel (core), from the live per-launch profile.
    det_ms = [ms for p in profs for ms in p["core_ms"]]
    per_kernel = {name: sum(ms for p in profs for ms in p[name + "_ms"])
                  for name in ("core", "grow")}
    per_kernel["final"] = sum(p["final_ms"] for p in profs)
    n_launch = len(det_ms)
    ops = sum(netcost.detect_minmax_ops(p) for p in profs)
    det_avg_ms = sum(det_ms) / max(1, n_launch)
    achieved = ops / n_launch / (det_avg_ms * 1e-3) / 1e12 if n_launch else None
    peak_f32, peak_u16 = alu_peak()
    peak = peak_f32 / 1e3 if peak_f32 else None
    share = per_kernel["core"] / sum(per_kernel.values())
    # End to end through the public API: lacos_submit_host copies the pinned
    # host frame in and the mask and cleaned frame out inside every step;
    # E2E_DEPTH requests in flight overlap one step's upload, another's
    # compute and a third's download.
    h_frame = torch.from_numpy(frame.view(np.int16)).pin_memory().view(torch.uint16)
    h_masks = [torch.empty((ny, nx), dtype=torch.uint8).pin_memory() for _ in range(E2E_DEPTH)]
    h_cleans = [torch.empty((ny, nx), dtype=torch.float32).pin_memory() for _ in range(E2E_DEPTH)]

    def e2e_run(n):
        return lacos.clean_host_stream(ctx, [h_frame] * n, params, [h_masks[i % E2E_DEPTH] for i in range(n)],
                                       [h_cleans[i % E2E_DEPTH] for i in range(n)], depth=E2E_DEPTH)

    e2e_run(E2E_DEPTH)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e2e_res = e2e_run(args.e2e_steps)
    torch.cuda.synchronize()
    e2e_s = pdist.max_over_ranks(time.perf_counter() - t0, dev)
    e2e_value = pdist.job_throughput(npix, args.e2e_steps, ws, e2e_s)

    last = (args.e2e_steps - 1) % E2E_DEPTH
    keep = h_masks[last].numpy() == 0
    ok_check = bool(all(r.status == 0 for r in e2e_res) and
                    np.array_equal(h_cleans[last].numpy()[keep], frame[keep].astype(np.float32)))
    ctx.close()
    del d_frame, d_mask, d_clean, flush
    torch.cuda.empty_cache()
    batched = serving = None
    if ws == 1 and not args.no_batched:
        batched = run_batched(args, dev)
    if ws == 1 and not args.no_serving:
        serving = run_serving(args, dev)
    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline else oracle_sample(frame, spec)
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(step_ms) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "ny": ny, "nx": nx, "frame_dtype": "u16", "niter": spec.niter,
                   "frames_per_call": 1, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tminmax/s",
                     "frac": (achieved / peak) if (achieved and peak) else None,
                     "traffic": NCU_CORE_TRAFFIC.get(kernel_source_sha()),
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read+write)",
                     "kernel": "core_kernel", "peak_source": "measured min.f32/max.f32 issue rate",
                     "avg_launch_ms": det_avg_ms, "launch_share": share,
                     "kernel_ms_per_step": {k: v / len(profs) for k, v in per_kernel.items()}},
        "e2e": {"value": e2e_value, "unit": "Mpix/s", "h2d_bytes_per_step": 2 * npix,
                "d2h_bytes_per_step": 5 * npix, "api": "lacos_submit_host",
                "requests_in_flight": E2E_DEPTH},
        "gpu_launches": args.steps * (2 * spec.niter + 2),
        "clocks": clk.summary(),
        "wall_s_timed": t_wall,
        "check_clean_equals_input_outside_mask": ok_check,
        "alu_peak_gops": {"f32": peak_f32, "u16x2": peak_u16},
        "sparse_work_per_step": {k: profs[-1][k] for k in ("n_sprime", "n_fine", "n_replace", "n_replace_wide")},
        "modes": modes,
    }
    line["core_variant"] = {"chosen": variant, "ms_per_variant": variant_ms}
    if batched:
        line["batched"] = batched
    if serving:
        line["serving"] = serving
        sat = serving["points"][0]
        line["p99_latency_ms"] = sat["p99_ms"]
        line["p99_latency_at"] = f"{sat['rate_hz']} frames/s Poisson, 120 GB budget"
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
