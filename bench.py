#!/usr/bin/env python3
"""Throughput of the FTK pose-scoring path on GB300.

One step = transform of every image and template (Fourier--Bessel coefficients)
plus the all-pairs search for each image's best (template, rotation, shift),
inputs resident in device memory. The metric counts pose inner products:
pairs x rotations (2Q) x shifts (N) per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision auto|fp32|bf16x3|bf16] [--workload n64_1k|n128_8k|batch4|...]
                  [--no-e2e] [--no-cpu-baseline] [--no-fp32] [--no-proposal] [--autotune] [--step23 0|1] [--eps E] [--decay B]
                  [--proposal-only] [--proposal-workload n64_prop] [--proposal-net shared|head|cnn16] [--proposal-k 128]
                  [--proposal-train 8192] [--proposal-eval 2048] [--proposal-epochs E]

After the timed region, rank 0 of a one-GPU run also times the same step on the
FP32 engine ("fp32_ftk") and the learned proposal path against the full search
on the proposal workload ("proposal"); neither is part of the headline value.

Under torchrun (N > 1) every rank runs the same per-GPU workload on its own
images (weak scaling, no collective on the data path); rank 0 prints one JSON line.
The CPU oracle is imported only for the cpu_baseline leg and the reference arm.
"""

from __future__ import annotations

import argparse
import hashlib
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

import numpy as np  # noqa: E402

METRIC = "pose inner products/sec (pairs x rotations x shifts) at stated eps vs FP32 FTK"
UNIT = "poses/s"
DEFAULT_WORKLOAD = "n128_8k"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
SMS = 152
FP32_LANES_PER_SM = 128


def rank_seed(rank: int):
    """Images are sharded across ranks: rank 0 uses the workload's own seed, the others their own."""
    return None if rank == 0 else 7000 + rank


def max_over_ranks(seconds: float, world: int, device=None) -> float:
    """The job's time is the slowest rank's (all_reduce MAX; no-op for one process)."""
    if world <= 1:
        return float(seconds)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step: float, steps: int, world: int, seconds: float) -> float:
    """Whole-job rate: every rank processes its own units (weak scaling)."""
    return world * units_per_rank_step * steps / seconds


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return dict(PEAKS_FALLBACK), "fallback"


def describe(wl, eps):
    return (f"{wl.name}: {wl.images.shape[0]} images x {wl.templates.shape[0]} templates, n={wl.n}, "
            f"M={wl.M}, 2Q={wl.two_Q}, N={wl.shifts_px.shape[0]}, eps={eps:g}, W={wl.W:g}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def l2_flusher(torch, device):
    buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=device)

    def flush():
        buf.zero_()
    return flush


def kernel_work(name, plan, wl, terms=None):
    """Algorithmic work per step of the named kernel: ("flops"|"bytes", amount).

    Per pair, with H the plan's rank over all Bessel orders (the algorithmic count of
    eq. fbk3): Step 3 = 4 N H 2Q flops (Re(Y Z), 2 real MACs per term); Step 1 =
    8 H M 2Q flops (one complex MAC per (zeta, q, m)); Step 2 + packing moves Zhat in
    (8 B per complex) and (Re Z, Im Z) out as bf16 hi/lo (8 B per complex).
    terms="executed" counts the H' = H_half terms of orders l >= 0 that the kernels
    evaluate instead: for real images the terms of order -l are the conjugates of those
    of order l, so the kernels do about half the algorithmic flops.
    The fused Steps 2-3 kernels are counted by their contraction (the Step-3 flops): the
    DFT over q adds 5 H' 2Q log2(2Q) flops on the FP32 pipes, not the tensor cores.
    """
    NI, NT = wl.images.shape[0], wl.templates.shape[0]
    pairs = NI * NT
    N, two_Q, M = plan.N, plan.two_Q, plan.M
    H = plan.H_half if terms == "executed" else plan.H
    Hh = plan.H_half
    if name in ("step3_simt", "step3_tc", "step23_tc", "step23c_tc"):
        return "flops", pairs * N * two_Q * 4 * H
    if name in ("step1_simt", "step1_tc"):
        return "flops", pairs * two_Q * H * M * 8
    if name == "fft_pack":
        return "bytes", pairs * Hh * two_Q * (8 + 8)
    if name == "fft_rows":
        return "bytes", pairs * Hh * two_Q * (8 + 8)
    return None, None


def src_hash(kernel):
    files = {"step3_simt": "k_simt.cu", "step1_simt": "k_simt.cu", "step3_tc": "k_tc.cu", "step1_tc": "k_tc_step1.cu",
             "fft_rows": "k_transform.cu", "polar_transform": "k_transform.cu", "fft_pack": "k_tc.cu",
             "polar_tc": "k_transform_tc.cu", "step23_tc": "k_step23_tc.cu"}
    f = files.get(kernel)
    if not f:
        return None
    with open(os.path.join(ROOT, "paper_1905_12317_gb300", "csrc", f), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def ncu_traffic(kernel, pairs_per_launch, grid):
    """DRAM bytes per launch from the committed ncu summaries: the entry taken on the same grid
    (n, 2Q, N), scaled from its pairs to the launch's, if the kernel source is unchanged since."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            tab = json.load(f)
    except Exception:
        return None
    for ent in tab.get(kernel, []):
        if (ent.get("grid") == grid and ent.get("src_sha") == src_hash(kernel)
                and "dram_bytes_per_pair" in ent):
            return ent["dram_bytes_per_pair"] * pairs_per_launch
    return None


def run_ours(args, rank, world, torch):
    import paper_1905_12317_gb300 as ftk
    from workloads import make_workload

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = make_workload(args.workload, seed=rank_seed(rank))
    eps = args.eps if args.eps else wl.eps
    plan = ftk.Plan(wl.n, wl.W, eps, wl.M, wl.two_Q, wl.shifts_px, decay=args.decay)
    prec_name = args.precision
    if prec_name == "auto":
        prec_name = "fp32"
        for cand in ("bf16x3",):
            try:
                z = torch.zeros((1, wl.M, wl.two_Q), dtype=torch.complex64, device=dev)
                plan.align_best(z, z, ftk.PRECISIONS[cand])
                torch.cuda.synchronize()
                prec_name = cand
                break
            except ftk.FtkError:
                pass
    prec = ftk.PRECISIONS[prec_name]
    NI, NT = wl.images.shape[0], wl.templates.shape[0]
    imgs = torch.from_numpy(np.ascontiguousarray(wl.images)).to(dev)
    tpls = torch.from_numpy(np.ascontiguousarray(wl.templates)).to(dev)
    a = torch.empty((NI, wl.M, wl.two_Q), dtype=torch.complex64, device=dev)
    b = torch.empty((NT, wl.M, wl.two_Q), dtype=torch.complex64, device=dev)
    _, gd = plan.workspace_size(prec, NI, NT)
    work = torch.empty(gd, dtype=torch.uint8, device=dev)
    outs = (torch.empty(NI, dtype=torch.int32, device=dev), torch.empty(NI, dtype=torch.int32, device=dev),
            torch.empty(NI, dtype=torch.int32, device=dev), torch.empty(NI, dtype=torch.float32, device=dev))
    stream = torch.cuda.current_stream()
    flush = l2_flusher(torch, dev)

    def step():
        plan.transform(imgs, out=a)
        plan.transform(tpls, out=b)
        plan.align_best(a, b, prec, work=work, out=outs)

    if prec_name != "fp32":
        plan.tune("step23", args.step23)   # 0: the separate Step-2 and Step-3 kernels
        plan.tune("cluster23", args.cluster23)
    tuned = None
    if args.autotune and prec_name != "fp32":
        from paper_1905_12317_gb300.autotune import autotune
        plan.transform(imgs, out=a)
        plan.transform(tpls, out=b)
        log = []
        tuned = autotune(plan, a, b, prec, work=work, log=log)
        for row in log:
            print("autotune", *row, file=sys.stderr)

    for _ in range(args.warmup):
        flush()
        step()
    plan.stream_check()
    torch.cuda.synchronize()

    clocks = ClockSampler(dev.index)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = plan.launch_count
    plan.profile_begin()
    evs = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    prof = plan.profile_end()
    launches = plan.launch_count - launches0
    plan.stream_check()
    clk = clocks.stop()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, dev)

    poses_step = NI * NT * wl.two_Q * wl.shifts_px.shape[0]
    value = job_throughput(poses_step, args.steps, world, total_s)

    # roofline of the dominant kernel
    peaks, peak_src = load_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][0])[0] if prof else None
    roof = None
    if dom:
        ms, nl = prof[dom]
        kind, amount = kernel_work(dom, plan, wl)
        if kind == "bytes":
            achieved = amount * args.steps / (ms / 1e3) / 1e9
            peak = peaks["hbm_gbs"]
            roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "peak_note": f"HBM copy bandwidth ({peak_src})"}
        elif kind == "flops":
            flops = amount
            achieved = flops * args.steps / (ms / 1e3) / 1e12
            executed = kernel_work(dom, plan, wl, terms="executed")[1] * args.steps / (ms / 1e3) / 1e12
            if dom.endswith("_tc"):
                mult = 3 if prec_name == "bf16x3" else 1
                peak = peaks["bf16_tflops"] / mult
                roof = {"bound": "tensor", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                        "frac": round(achieved / peak, 4),
                        "peak_note": f"bf16 burst of {peak_src} / {mult} MMAs per product"
                                     + (" (fp16 runs at the bf16 dense rate)" if prec_name == "fp16" else ""),
                        "work_note": "achieved = 4 N H 2Q flops per pair (H = rank over all orders, the "
                                     "algorithmic count of eq. fbk3); executed = the same with H' = terms of orders l >= 0, which "
                                     "the kernels evaluate",
                        "executed": round(executed, 3), "executed_frac": round(executed / peak, 4)}
            else:
                peak = SMS * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
                roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                        "frac": round(achieved / peak, 4),
                        "peak_note": "FP32 FFMA: 152 SMs x 128 lanes x 2 flops x max SM clock"}
        if roof is not None:
            pairs_per_launch = NI * NT * args.steps / nl
            # the committed counters are of the plain plan: a weighted plan has fewer terms (a smaller Zhat)
            grid = {"n": wl.n, "two_Q": wl.two_Q, "N": int(wl.shifts_px.shape[0])}
            roof["traffic"] = ncu_traffic(dom, pairs_per_launch, grid) if not plan.decay else None
            roof["kernel"] = dom
            roof["avg_launch_ms"] = round(ms / nl, 4)
    shares = {k: round(v[0] / sum(x[0] for x in prof.values()), 4) for k, v in prof.items()} if prof else {}

    # end to end through the public C ABI from host buffers
    e2e = None
    if not args.no_e2e:
        h_imgs = torch.from_numpy(np.ascontiguousarray(wl.images)).pin_memory()
        h_tpls = torch.from_numpy(np.ascontiguousarray(wl.templates)).pin_memory()
        _, sgd = plan.search_workspace_size(prec, NI, NT)
        swork = torch.empty(sgd, dtype=torch.uint8, device=dev)
        hout = tuple(torch.empty(NI, dtype=d).pin_memory()
                     for d in (torch.int32, torch.int32, torch.int32, torch.float32))
        for _ in range(2):
            plan.search_host(h_imgs, h_tpls, prec, swork, hout)
        times = []
        reps = min(args.steps, 5)  # each rep is one full step from host buffers
        for _ in range(reps):
            flush()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            plan.search_host(h_imgs, h_tpls, prec, swork, hout)
            times.append(time.perf_counter() - t1)
        e2e = {"value": job_throughput(poses_step, reps, world, max_over_ranks(sum(times), world, dev)),
               "unit": UNIT, "steps": reps,
               "h2d_bytes_per_step": int((NI + NT) * wl.n * wl.n * 4), "d2h_bytes_per_step": int(NI * 16)}

    return dict(value=value, total_s=total_s, step_ms=step_ms, wall=wall, prec=prec_name, wl=wl, eps=eps, plan=plan,
                roof=roof, shares=shares, prof=prof, launches=launches, clocks=clk, e2e=e2e, outs=outs,
                tuned=tuned if tuned is not None else (plan.tuning() if prec_name != "fp32" else None))


def run_batch(args, torch):
    """The uneven-groups workload: four image sizes, each group against its own templates, one step
    = transforms + best-pose search of every group, replayed as one CUDA graph."""
    import paper_1905_12317_gb300 as ftk
    from paper_1905_12317_gb300.batch import Group, GroupedSearch
    from workloads import BATCH_GROUPS, make_workload
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    prec_name = "bf16x3" if args.precision == "auto" else args.precision
    prec = ftk.PRECISIONS[prec_name]
    wls, groups, tuned = [], [], {}
    for name in BATCH_GROUPS:
        wl = make_workload(name)
        plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
        g = Group(plan=plan, images=torch.from_numpy(wl.images).to(dev),
                  templates=torch.from_numpy(wl.templates).to(dev), precision=prec)
        wls.append(wl)
        groups.append(g)
    gs = GroupedSearch(groups, device=dev)
    if prec_name != "fp32":  # tile shapes per group from the autotuner
        from paper_1905_12317_gb300.autotune import autotune
        for wl, g in zip(wls, gs.groups):
            g.plan.transform(g.images, out=g.a)
            g.plan.transform(g.templates, out=g.b)
            tuned[wl.name] = autotune(g.plan, g.a, g.b, prec, work=g.work)
    flush = l2_flusher(torch, dev)
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        for _ in range(args.warmup):
            flush()
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            ms.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ms]

    seq = timed(lambda: gs.step_eager(concurrent=False), args.steps)
    conc = timed(lambda: gs.step_eager(concurrent=True), args.steps)
    # launches of one step, counted on the eager path (a graph replay runs the same kernels)
    l0 = sum(g.plan.launch_count for g in gs.groups)
    gs.step_eager(concurrent=True)
    per_step = sum(g.plan.launch_count for g in gs.groups) - l0
    gs.capture()
    clocks = ClockSampler(dev.index)
    clocks.start()
    graph = timed(gs.replay, args.steps)
    clk = clocks.stop()
    for g in gs.groups:
        g.plan.stream_check()
    poses = gs.poses_per_step()
    total_s = sum(graph) / 1e3
    value = poses * args.steps / total_s

    # roofline of the dominant kernel over all groups (a profiled sequential step)
    for g in gs.groups:
        g.plan.profile_begin()
    gs.step_eager(concurrent=False)
    profs = [g.plan.profile_end() for g in gs.groups]
    agg = {}
    for pf in profs:
        for k, (ms, n) in pf.items():
            agg[k] = (agg.get(k, (0.0, 0))[0] + ms, agg.get(k, (0.0, 0))[1] + n)
    dom = max(agg.items(), key=lambda kv: kv[1][0])[0]
    peaks, peak_src = load_peaks()
    kinds = [kernel_work(dom, g.plan, wl) for g, wl in zip(gs.groups, wls)]
    amount = sum(a for _, a in kinds if a)
    kind = kinds[0][0]
    roof = None
    if kind == "flops" and dom.endswith("_tc"):
        mult = 3 if prec_name == "bf16x3" else 1
        achieved = amount / (agg[dom][0] / 1e3) / 1e12
        peak = peaks["bf16_tflops"] / mult
        roof = {"bound": "tensor", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "peak_note": f"bf16 burst of {peak_src} / {mult} MMAs per product",
                "traffic": None, "kernel": dom, "avg_launch_ms": round(agg[dom][0] / agg[dom][1], 4)}
    elif kind == "bytes":
        achieved = amount / (agg[dom][0] / 1e3) / 1e9
        peak = peaks["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_note": f"HBM copy bandwidth ({peak_src})", "traffic": None,
                "kernel": dom, "avg_launch_ms": round(agg[dom][0] / agg[dom][1], 4)}
    tot = sum(v[0] for v in agg.values())
    shares = {k: round(v[0] / tot, 4) for k, v in agg.items()}

    e2e = None
    if not args.no_e2e:
        hosts = [(torch.from_numpy(wl.images).pin_memory(), torch.from_numpy(wl.templates).pin_memory()) for wl in wls]
        works, houts = [], []
        for g, (hi, ht) in zip(gs.groups, hosts):
            works.append(torch.empty(g.plan.search_workspace_size(prec, hi.shape[0], ht.shape[0])[1],
                                     dtype=torch.uint8, device=dev))
            houts.append(tuple(torch.empty(hi.shape[0], dtype=d).pin_memory()
                               for d in (torch.int32, torch.int32, torch.int32, torch.float32)))

        def host_step():
            for g, (hi, ht), w, ho in zip(gs.groups, hosts, works, houts):
                g.plan.search_host(hi, ht, prec, w, ho)
        host_step()
        times = []
        for _ in range(args.steps):
            flush()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            host_step()
            times.append(time.perf_counter() - t1)
        e2e = {"value": poses * args.steps / sum(times), "unit": UNIT,
               "h2d_bytes_per_step": int(sum((wl.images.shape[0] + wl.templates.shape[0]) * wl.n * wl.n * 4
                                             for wl in wls)),
               "d2h_bytes_per_step": int(sum(wl.images.shape[0] * 16 for wl in wls))}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(BATCH_GROUPS[0], args.cpu_budget)
    desc = "; ".join(f"{wl.name}: {wl.images.shape[0]}x{wl.templates.shape[0]}, n={wl.n}, 2Q={wl.two_Q}, "
                     f"N={wl.shifts_px.shape[0]}, H={g.plan.H}" for wl, g in zip(wls, gs.groups))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(graph) / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16x3": "bf16x3 (fp32 accumulate)", "bf16": "bf16 (fp32 accumulate)",
                  "fp16": "f16 (fp32 accumulate)"}[prec_name],
        "data": "synthetic",
        "config": {"workload": f"batch4 (uneven groups, eps=1e-3): {desc}", "precision": prec_name,
                   "step": "per group: transform(images)+transform(templates)+align_best; groups on own streams, "
                           "one CUDA graph replay",
                   "l2": "flushed between timed steps (512 MiB device write)", "parallelism": "single GPU",
                   "launch_shapes": tuned or {wl.name: g.plan.tuning() for wl, g in zip(wls, gs.groups)}},
        "sequential_launches_ms_per_step": round(sum(seq) / args.steps, 3),
        "concurrent_streams_ms_per_step": round(sum(conc) / args.steps, 3),
        "roofline": roof, "kernel_shares": shares, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": per_step * args.steps, "clocks": clk,
    }
    print(json.dumps(line))


def cuda_ms(torch, fn, reps=3):
    """Average device time of fn() over reps calls (CUDA events on the current stream, after one warm call)."""
    out = fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def fp32_compare(torch, r, steps=1, budget_s=4.0, rate_guess=7e10):
    """The same step (transforms + all-pairs best pose) on the FP32 SIMT engine, same GPU and
    inputs, on a sample of the images (about budget_s seconds at rate_guess poses/s) against
    all templates; the rate is per pose, so it compares directly with the headline."""
    import paper_1905_12317_gb300 as ftk
    plan, wl = r["plan"], r["wl"]
    dev = torch.device("cuda", torch.cuda.current_device())
    NI, NT = wl.images.shape[0], wl.templates.shape[0]
    per_image = NT * wl.two_Q * wl.shifts_px.shape[0]
    ni = int(max(1, min(NI, rate_guess * budget_s // per_image)))
    imgs = torch.from_numpy(np.ascontiguousarray(wl.images[:ni])).to(dev)
    tpls = torch.from_numpy(np.ascontiguousarray(wl.templates)).to(dev)
    work = torch.empty(plan.workspace_size(ftk.FP32, ni, NT)[1], dtype=torch.uint8, device=dev)

    def step():
        a, b = plan.transform(imgs), plan.transform(tpls)
        return plan.align_best(a, b, ftk.FP32, work=work)

    ms, out = cuda_ms(torch, step, reps=steps)
    agree = float((out[0] == r["outs"][0][:ni]).double().mean())
    v = ni * per_image / (ms / 1e3)
    return {"value": v, "unit": UNIT, "ms_per_step": round(ms, 2), "speedup_of_headline": round(r["value"] / v, 2),
            "sample": f"{ni} of {NI} images x all {NT} templates (transforms included)",
            "best_template_agreement": round(agree, 4)}


def proposal_leg(torch, workload="n64_prop", net="shared", n_train=8192, n_eval=2048, epochs=None, K=128,
                 target=0.995):
    """Learned proposal path (trained here on FTK labels) against the full search.

    net: "shared" = template head whose analytic FTK filters share one learned spectral weight
    (the default); "head" = template head with every template's filter learned; "cnn16" = the
    per-template head + CNN branch 16/32/32/32 with an MLP of 128.
    """
    import paper_1905_12317_gb300 as ftk
    from paper_1905_12317_gb300 import proposal as pr
    from workloads import CONFIGS, make_workload
    dev = torch.device("cuda", torch.cuda.current_device())
    cfg = CONFIGS[workload]
    tr = make_workload(workload, n_images=n_train, noise=False)
    te = make_workload(workload, n_images=2 * n_eval, image_seed=1)
    plan = ftk.Plan(tr.n, tr.W, tr.eps, tr.M, tr.two_Q, tr.shifts_px)
    _, wr = plan.radial_rule()
    clean = torch.from_numpy(tr.images).to(dev)
    sd = torch.sqrt((clean * clean).mean(dim=(1, 2)) / cfg["snr"])[:, None, None]
    b = plan.transform(torch.from_numpy(tr.templates).to(dev))
    NT = b.shape[0]
    shifts = torch.from_numpy(tr.shifts_px.astype(np.float32)).to(dev)
    rings, band = 3 * tr.M // 8, tr.two_Q // 4
    kw = dict(cnn=False, head_weight="shared") if net == "shared" else (
        dict(cnn=False) if net == "head" else dict(ch=(16, 32, 32, 32), hidden=128))
    lr = 3e-2 if net == "shared" else 1e-3
    epochs = epochs or (8 if net == "shared" else 6)
    model = pr.ProposalNet(tr.M, tr.two_Q // 2, NT, head_rings=rings, head_band=band, seed=0, **kw)
    gen = torch.Generator(device=dev).manual_seed(1000)
    a0 = plan.transform(clean[:256] + sd[:256] * torch.randn((256,) + clean.shape[1:], generator=gen, device=dev))
    model.init_head(b, wr, a_sample=a0)
    at = plan.transform(torch.from_numpy(te.images).to(dev))
    aev0 = at[n_eval:].contiguous()
    ft0 = plan.align_best(aev0, b, ftk.BF16X3)[0]
    ks = sorted({1, 4, 16, K})
    recall_init = {k: round(pr.recall_at_k(model.propose(aev0, k)[0], ft0), 4) for k in ks}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = pr.train_with_ftk_labels(plan, model, b, clean, sd, shifts, epochs, lr=lr)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    recall_trained = {k: round(pr.recall_at_k(model.propose(aev0, k)[0], ft0), 4) for k in ks}
    at = plan.transform(torch.from_numpy(te.images).to(dev))
    acal, aev = at[:n_eval].contiguous(), at[n_eval:].contiguous()
    wsl = torch.empty(pr.shortlist_workspace_size(plan, ftk.BF16X3, n_eval, NT, K)[1], dtype=torch.uint8,
                      device=dev)
    thr = pr.calibrate_path(plan, model, acal, b, K, target, work=wsl)
    wfull = torch.empty(plan.workspace_size(ftk.BF16X3, n_eval, NT)[1], dtype=torch.uint8, device=dev)
    t_full, full = cuda_ms(torch, lambda: plan.align_best(aev, b, ftk.BF16X3, work=wfull))
    ft, fr, fs = (x.clone() for x in full[:3])
    t_path, (res, n_fb) = cuda_ms(torch, lambda: pr.search_with_proposals(plan, model, aev, b, k=K, min_conf=thr,
                                                                          precision=ftk.BF16X3, work=wsl))
    same = float(((res[0] == ft) & (res[1] == fr) & (res[2] == fs)).double().mean())
    recall_k = pr.recall_at_k(model.propose(aev, K)[0], ft)
    poses = n_eval * NT * tr.two_Q * tr.shifts_px.shape[0]
    return {"workload": f"{workload}: {n_eval} images x {NT} templates (centred), n={tr.n}, M={tr.M}, "
                        f"2Q={tr.two_Q}, N={tr.shifts_px.shape[0]}, eps={tr.eps:g}, SNR {cfg['snr']:g}",
            "network": (f"rotation-equivariant template head ({rings} rings, |q|<={band})" +
                        {"shared": ", analytic FTK filters with one learned spectral weight",
                         "head": ", every template's filter learned",
                         "cnn16": ", every template's filter learned, + CNN 16/32/32/32 + MLP 128"}[net] +
                        ", FP32 CUDA forward/backward/Adam"),
            "train": {"images": n_train * epochs, "epochs": epochs, "lr": lr, "labels": "full FTK search, bf16x3",
                      "seconds": round(train_s, 2), "loss_first_last": [round(losses[0], 4), round(losses[-1], 4)]},
            "recall_at_k_before_training": recall_init, "recall_at_k_after_training": recall_trained,
            "k": K, "recall_at_k": round(recall_k, 4), "calibration_target": target,
            "min_shortlist_mass": round(thr, 4), "fallback_frac": round(n_fb / n_eval, 4),
            "path_recall_of_full_search_pose": round(same, 4), "path_ms": round(t_path, 2),
            "full_search_ms": round(t_full, 2), "speedup": round(t_full / t_path, 2),
            "equivalent_poses_per_s": poses / (t_path / 1e3)}


_ORACLE = {}   # per spawned host process: the oracle's inputs, built once (_oracle_init)


def _oracle_init(workload: str, per: int, eps: float | None = None):
    """Pool initializer: one image and `per` templates of the workload's recipe (a seed of
    the process's own), their FP64 transforms, the FP64 plan and the shift vectors."""
    import multiprocessing as mp
    from oracle import brute, quadrature as quad, svd_plan, transform as tr
    from workloads import CONFIGS, make_workload

    ident = mp.current_process()._identity
    rank = ident[0] if ident else 0
    seed = 1905 + list(CONFIGS).index(workload) + 1000 * rank
    wl = make_workload(workload, seed=seed, n_images=1, n_templates=per)
    K = quad.nyquist_K(wl.n)
    k, w = quad.radial_rule(wl.M, K)
    _ORACLE.update(a=tr.fourier_bessel(wl.images.astype(np.float64), k, wl.two_Q),
                   b=tr.fourier_bessel(wl.templates.astype(np.float64), k, wl.two_Q), k=k, w=w,
                   plan=svd_plan.build_plan(wl.W, eps or wl.eps, K), delta=brute.shift_vectors(wl.shifts_px, wl.n),
                   poses=wl.two_Q * wl.shifts_px.shape[0])


def _oracle_timed(budget_s: float):
    """Scores pairs with the FP64 step-by-step oracle (O2) for about budget_s seconds."""
    from oracle import ftk_steps
    o = _ORACLE
    done = 0
    t0 = time.perf_counter()
    nb = o["b"].shape[0]
    while time.perf_counter() - t0 < budget_s:   # the process's templates in turn
        j = done % nb
        ftk_steps.ftk_scores(o["a"][0], o["b"][j:j + 1], o["k"], o["w"], o["plan"], o["delta"])
        done += 1
    return done, time.perf_counter() - t0, o["poses"]


_POOLS = {}


def _oracle_pool(workload: str, n: int, per: int, eps: float | None = None):
    """One pool of host processes per workload for the whole run (started with spawn, so it is
    safe after CUDA work in this process); the inputs are built once per process."""
    import atexit
    import multiprocessing as mp
    key = (workload, n, per, eps)
    if key not in _POOLS:
        # one core per process: the spawned interpreters start with single-threaded BLAS
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        os.environ.update({v: "1" for v in saved})
        try:
            pool = mp.get_context("spawn").Pool(n, initializer=_oracle_init, initargs=(workload, per, eps))
        finally:
            for v, x in saved.items():
                if x is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = x
        atexit.register(pool.terminate)
        _POOLS[key] = pool
    return _POOLS[key]


def cpu_oracle_rate(workload: str, budget_s: float, processes: int | None = None, eps: float | None = None):
    """FP64 oracle (step-by-step FTK, as written) on the host cores: one process per core, each
    scoring one image against its own templates of the workload's recipe for about budget_s
    seconds (plan and transforms built once per process and excluded)."""
    n = processes or max(1, os.cpu_count() or 1)
    per = 4  # templates per process, scored in turn (the oracle's time per pair does not depend on them)
    res = _oracle_pool(workload, n, per, eps).map(_oracle_timed, [budget_s] * n)
    done = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    poses_per_pair = res[0][2]
    return {"value": done * poses_per_pair / wall, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"FP64 step-by-step FTK oracle (numpy), {n} processes x 1 image x {per} templates "
                      f"of the {workload} recipe{f' at eps {eps:g}' if eps else ''} scored in turn ({done} pairs), plan and transforms excluded, "
                      f"{wall:.1f} s wall"}


def run_reference(args) -> dict:
    """The reference arm: the FP64 oracle on the host cores, each step a bounded sample of the
    workload (cpu_oracle_rate), reported on the metric and unit of the GPU arm."""
    per_step = []
    base = None
    from workloads import BATCH_GROUPS, CONFIGS, make_workload
    wname = BATCH_GROUPS[0] if args.workload == "batch4" else args.workload
    eps = getattr(args, "eps", None)  # the plan's precision target where overridden
    for it in range(args.warmup + args.steps):
        r = cpu_oracle_rate(wname, budget_s=max(2.0, 60.0 / (args.warmup + args.steps)), eps=eps)
        if it >= args.warmup:
            per_step.append(r["value"])
        base = r
    wl = make_workload(wname, n_images=1, n_templates=1)
    cfg = CONFIGS[wname]
    v = statistics.mean(per_step)
    poses_step = cfg["n_images"] * cfg["n_templates"] * wl.two_Q * wl.shifts_px.shape[0]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": poses_step / v * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(wl, eps or wl.eps).replace(
                           "1 images x 1 templates", f"{cfg['n_images']} images x {cfg['n_templates']} templates"),
                       "sample": base["sample"],
                       "ms_per_step": "one full step of the workload at the sampled rate (extrapolated)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16x3", "bf16", "fp16"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--autotune", action="store_true", help="pick launch shapes with the autotuner before timing")
    ap.add_argument("--step23", type=int, default=1, choices=[0, 1],
                    help="1: Steps 2-3 fused where the plan fits (default); 0: the separate Step-2 and Step-3 kernels")
    ap.add_argument("--cluster23", type=int, default=0, choices=[0, 1],
                    help="1: Steps 2-3 fused over a CTA cluster where 2Q = 128 R; 0: separate kernels there (default)")
    ap.add_argument("--eps", type=float, default=None,
                    help="precision target of the plan (default: the workload's, 1e-3; config 3 also names 1e-4)")
    ap.add_argument("--decay", type=float, default=0.0,
                    help="spectral weight exp(-decay (k/K)^2) of the plan's SVDs (ftk_plan_create_weighted); "
                         "0: the plain plan (default)")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-engine comparison")
    ap.add_argument("--no-proposal", action="store_true", help="skip the learned-proposal leg")
    ap.add_argument("--proposal-only", action="store_true",
                    help="run only the learned-proposal leg and print its JSON object")
    ap.add_argument("--proposal-workload", default="n64_prop")
    ap.add_argument("--proposal-net", default="shared", choices=["shared", "head", "cnn16"])
    ap.add_argument("--proposal-k", type=int, default=128)
    ap.add_argument("--proposal-train", type=int, default=8192, help="training images per epoch")
    ap.add_argument("--proposal-eval", type=int, default=2048, help="calibration and evaluation images (each)")
    ap.add_argument("--proposal-epochs", type=int, default=0, help="0: the network's default")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 0)

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args)))
        return

    import torch
    if args.proposal_only:
        if rank == 0:
            print(json.dumps(proposal_leg(torch, args.proposal_workload, args.proposal_net, n_train=args.proposal_train,
                                          n_eval=args.proposal_eval, epochs=args.proposal_epochs or None,
                                          K=args.proposal_k)))
        return
    if args.workload == "batch4":
        if rank == 0:
            run_batch(args, torch)
        return
    if world > 1:
        torch.distributed.init_process_group("nccl")
    r = run_ours(args, rank, world, torch)
    if rank == 0:
        wl, plan = r["wl"], r["plan"]
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_oracle_rate(args.workload, args.cpu_budget, eps=args.eps)
        fp32 = fp32_compare(torch, r) if (not args.no_fp32 and world == 1 and r["prec"] != "fp32") else None
        prop = (proposal_leg(torch, args.proposal_workload, args.proposal_net, K=args.proposal_k)
                if (not args.no_proposal and world == 1) else None)
        line = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["total_s"] * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16x3": "bf16x3 (fp32 accumulate)", "bf16": "bf16 (fp32 accumulate)",
                  "fp16": "f16 (fp32 accumulate)"}[r["prec"]],
            "data": "synthetic",
            "config": {"workload": describe(wl, r["eps"]), "n": wl.n, "M": wl.M, "two_Q": wl.two_Q,
                       "N": int(wl.shifts_px.shape[0]), "H": plan.H, "H_half": plan.H_half, "eps": r["eps"],
                       "precision": r["prec"], "step": "transform(images)+transform(templates)+align_best",
                       "l2": "flushed between timed steps (512 MiB device write)",
                       "parallelism": f"replicas x{world}, images sharded, templates replicated",
                       "steps_2_3": ("fused (k_step23_tc)" if "step23_tc" in r["shares"]
                                     else ("fused over 4-CTA clusters (k_step23c_tc)" if "step23c_tc" in r["shares"]
                                           else "separate (k_fft_pack, k_step3_tc)")),
                       "launch_shapes": r["tuned"],
                       **({"spectral_decay": args.decay} if args.decay else {})},
            "roofline": r["roof"], "kernel_shares": r["shares"], "cpu_baseline": cpu, "e2e": r["e2e"],
            "gpu_launches": r["launches"], "clocks": r["clocks"],
            "fp32_ftk": fp32, "proposal": prop,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
