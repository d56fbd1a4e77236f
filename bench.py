#!/usr/bin/env python3
"""Benchmark of C = lower(A·Aᵀ) mod p on GB300 (arXiv 2001.04109, Algorithm 2).

One "step" is one library call ffsyrk_with_plan on device-resident input:
digit split / pre-additions, every leaf product and the post-additions.  The
metric is the effective rate n²·k / t (the paper's effective-Gfops
definition with n³ → n²·k, counted once per output entry pair).

Prints one JSON line.  ``--impl reference`` times the CPU oracle (the
schoolbook definition) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "A·Aᵀ mod p effective ops/s (n²k/t), fast vs classical SYRK on 1 GB300, bit-exact"
UNIT = "ops/s"

WORKLOADS = {
    # name: (n, k, p, description)
    "square4096": (4096, 4096, 65521,
                   "A·Aᵀ mod p, A 4096×4096 uint32 uniform in [0,p), p=65521"),
    "small256": (256, 256, 65521, "A·Aᵀ mod p, A 256×256, p=65521"),
    "tall": (16384, 4096, 131071, "A·Aᵀ mod p, A 16384×4096, p=131071 (2×2 Y)"),
    "wide": (4096, 16384, 131071, "A·Aᵀ mod p, A 4096×16384, p=131071 (2×2 Y)"),
    "odd": (16383, 4097, 131071, "A·Aᵀ mod p, A 16383×4097, p=131071 (2×2 Y, padding)"),
    "square8192": (8192, 8192, 65521, "A·Aᵀ mod p, A 8192×8192, p=65521"),
    "square16384": (16384, 16384, 65521, "A·Aᵀ mod p, A 16384×16384, p=65521"),
    "large": (32768, 32768, 8388593, "A·Aᵀ mod p, A 32768×32768, p=8388593 (D=3)"),
}
DEFAULT_WORKLOAD = "large"
# 2048 independent problems, n and k each log-uniform in [32, 2048] (seed 5), p = 65521
BATCH = {"count": 2048, "lo": 32, "hi": 2048, "seed": 5, "p": 65521,
         "description": "batched A·Aᵀ mod p: 2048 problems, n, k log-uniform in [32, 2048], p=65521"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_source_hash(kernel_file: str):
    """sha256 (16 hex digits) of the kernel's source and the device helpers it includes."""
    csrc = os.path.join(ROOT, "paper_2001_04109_gb300", "csrc")
    h = hashlib.sha256()
    try:
        for name in (kernel_file, "tc_common.cuh"):
            h.update(open(os.path.join(csrc, name), "rb").read())
    except OSError:
        return None
    return h.hexdigest()[:16]


def plan_signature(info: dict, unit_bounds: str) -> str:
    """The plan choices a leaf's DRAM traffic depends on (not the epilogue warp count), as a
    profile's `plan:` line states them."""
    lv = info["levels"]
    wg = ",".join(str(x) for x in info["winograd"][:lv]) or "-"
    return (f"levels={lv} winograd={wg} tile_ctas={info['tile_ctas']} "
            f"products={info['products']} unit_bounds={unit_bounds}")


def kernel_traffic(kernel_file: str, workload: str, plan: str | None = None):
    """dram bytes per launch recorded under profiles/ for this kernel source (and, where the
    profile states one, this plan), else None."""
    h = kernel_source_hash(kernel_file)
    if h is None:
        return None
    prof = os.path.join(ROOT, "profiles")
    if not os.path.isdir(prof):
        return None
    for name in sorted(os.listdir(prof)):
        if not name.endswith((".txt", ".md")):
            continue
        text = open(os.path.join(prof, name)).read()
        m_src = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", text)
        m_wl = re.search(r"workload:\s*(\S+)", text)
        m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
        m_k = re.search(r"kernel_file:\s*(\S+)", text)
        m_plan = re.search(r"^plan:\s*(.+?)\s*$", text, re.M)
        if m_src and m_tr and m_k and m_wl and m_src.group(1) == h and m_k.group(1) == kernel_file \
                and m_wl.group(1) == workload and (m_plan is None or m_plan.group(1) == plan):
            return float(m_tr.group(1))
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    """The largest x over the ranks of the process group (x itself for one rank).

    Replicas time their own steps; the job's time is the slowest rank's.  The
    reduction runs on the GPU under NCCL and on the CPU under gloo.
    """
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(A_np, p, budget_s: float, keep_rows: bool = False):
    """Time the schoolbook oracle on a bounded row sample; effective n²k/s of the full product.

    The sample is rows spread evenly over A; their time is scaled (an
    extrapolation) to the n(n+1)/2 dot products of the lower triangle.  With
    ``keep_rows`` the sampled rows and their oracle values come back too,
    for the bit-exactness check of the GPU result.
    """
    import numpy as np

    import oracle
    n, k = A_np.shape
    threads = oracle.default_threads()
    rows_total = n
    # calibrate on a few rows, then size the sample to the budget
    r0 = max(1, min(n, threads))
    t0 = time.perf_counter()
    oracle.syrk_rows(A_np, p, np.arange(r0), threads=threads)
    t_cal = max(time.perf_counter() - t0, 1e-6)
    per_row = t_cal / r0
    r = int(max(r0, min(rows_total, budget_s / per_row)))
    rows = np.unique(np.linspace(0, n - 1, r).astype(np.int64))
    r = len(rows)
    t0 = time.perf_counter()
    vals = oracle.syrk_rows(A_np, p, rows, threads=threads)
    dt = time.perf_counter() - t0
    # a full row is n dot products; the lower product needs n(n+1)/2 of them
    t_full = dt / (r * n) * (n * (n + 1) / 2)
    out = {"value": n * n * k / t_full, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{r} full rows of A·Aᵀ mod p spread over A ({r * n} entries, {dt:.1f} s), "
                     f"time extrapolated to the {n}×{n} lower triangle"}
    if keep_rows:
        return out, rows, vals
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    from paper_2001_04109_gb300 import inputs
    if args.workload == "batched":
        count0 = args.batch_count or BATCH["count"]
        shapes = inputs.batch_shapes(count0, BATCH["lo"], BATCH["hi"], BATCH["seed"])
        vals, base = [], None
        for s in range(args.warmup + args.steps):
            r = cpu_batched_rate(shapes, BATCH["p"], args.ref_budget)
            if s >= args.warmup:
                vals.append(r["value"])
                base = r
        v = statistics.median(vals)
        ops = float(sum(n * n * k for n, k in shapes))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ops / v * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic", "config": {"workload": "batched",
                                                "description": BATCH["description"]},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": base["cores"],
                                 "kind": "oracle", "sample": base["sample"]},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    n, k, p, desc = WORKLOADS[args.workload]
    # the input is drawn on the GPU when there is one (same bits, much
    # faster for A 32768²); only the oracle's rows are timed
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A = inputs.uniform_residues(n, k, p, seed=2, device=dev).cpu().numpy().view(np.uint32)
    vals = []
    base = None
    for s in range(args.warmup + args.steps):
        r = cpu_oracle_rate(A, p, budget_s=args.ref_budget)
        if s >= args.warmup:
            vals.append(r["value"])
            base = r
    v = statistics.median(vals)
    ms = n * n * k / v * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": args.workload, "description": desc,
                                            "n": n, "k": k, "p": p},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_plan(plan, A, C, steps, warmup, flush, stream, timing=True):
    """Device time per call (CUDA events on the launching stream), L2 flushed between calls.

    The timed calls run exactly as a user's repeated calls do (the library
    replays its captured launch graph).  With ``timing``, a second pass of the
    same length records the library's per-stage events (direct launches) for
    the stage split and the leaf kernel's own duration.
    """
    import torch
    for _ in range(warmup):
        plan(A, C, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for s in range(steps):
        flush.zero_()
        ev[s][0].record(stream)
        plan(A, C, stream=stream)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    stage = []
    if timing:
        plan.set_timing(True)
        for s in range(steps):
            flush.zero_()
            plan(A, C, stream=stream)
            stage.append(plan.timing())
        torch.cuda.synchronize()
        plan.set_timing(False)
    return ms, stage


def golden_digest(n, k, p, seed=2):
    """The oracle's SHA-256 of the whole lower triangle, if tests/golden holds it."""
    path = os.path.join(ROOT, "tests", "golden", "fullsize_sha256.txt")
    try:
        for line in open(path):
            f = line.split()
            if len(f) == 5 and f[:4] == [str(n), str(k), str(p), str(seed)]:
                return f[4]
    except OSError:
        pass
    return None


def lower_digest(C_host):
    """SHA-256 of the lower triangle, rows in order, entries uint32 little-endian."""
    import numpy as np
    C = np.ascontiguousarray(C_host.numpy().view(np.uint32).astype("<u4", copy=False))
    h = hashlib.sha256()
    for i in range(C.shape[0]):
        h.update(C[i, : i + 1].tobytes())
    return h.hexdigest()


def describe(desc, info):
    """The workload's description with the depth and Winograd levels the plan took."""
    L = info["levels"]
    wg = info["winograd"][:L]
    if L == 0:
        how = "classical leaves only (depth 0)"
    else:
        how = f"Algorithm 2 at depth {L}"
        if any(wg):
            how += f", Algorithm 1 levels {wg} for the general products by depth"
    return f"{desc}; {how}"


def copy_ceiling(n, k, stream, reps=3):
    """Plain pinned-memory copies of one step's input (H2D) and result (D2H): ms each."""
    import torch
    a_h = torch.empty((n, k), dtype=torch.int32).pin_memory()
    c_h = torch.empty((n, n), dtype=torch.int32).pin_memory()
    a_d = torch.empty((n, k), dtype=torch.int32, device="cuda")
    c_d = torch.empty((n, n), dtype=torch.int32, device="cuda")
    out = {}
    for name, dst, src in (("h2d_ms", a_d, a_h), ("d2h_ms", c_h, c_d)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
        out[name] = statistics.median(t)
    del a_h, c_h, a_d, c_d
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2001_04109_gb300 import ffsyrk, inputs

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    __graft_entry__.build()
    n, k, p, desc = WORKLOADS[args.workload]
    levels = args.levels
    if levels is None and args.workload == "small256":
        levels = 0
    stream = torch.cuda.current_stream()
    # the same bits on host and device (counter-based generator); drawn on
    # the device, then copied, which is much faster for A 32768²
    A = inputs.uniform_residues(n, k, p, seed=2, device="cuda")
    A_host = A.cpu()
    C = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    # the default workload takes the plan's autotuner (depth, tiles, Winograd
    # levels, digit products timed at this size when the plan is made, outside
    # the timed region) unless options pin them
    autotune = args.autotune or (args.workload == DEFAULT_WORKLOAD and not args.no_autotune and
                                 levels is None and args.tile_ctas == 0 and args.winograd is None
                                 and args.digit_products == "auto" and args.leaf == "tc")
    t_plan = time.perf_counter()
    plan = ffsyrk.Plan(p, n, k, leaf=args.leaf, levels=levels, tile_ctas=args.tile_ctas,
                       winograd=args.winograd, digit_products=args.digit_products,
                       autotune=autotune, epilogue_warps=args.epilogue_warps,
                       unit_bounds=args.unit_bounds)
    plan_s = time.perf_counter() - t_plan
    info = plan.info()
    # the options that reproduce the plan's (tuned) choice, for the other plans of this run
    wl = info["winograd"][: info["levels"]]
    # the Winograd option that gives these levels: a cap w (min(w, L − 1 − d) at
    # depth d), else the cost model's choice, else none
    caps = [w for w in (1, 2, 3) if wl == [min(w, info["levels"] - 1 - d) for d in range(len(wl))]]
    same_opts = dict(leaf=args.leaf, levels=info["levels"], tile_ctas=info["tile_ctas"],
                     winograd=caps[0] if caps else (None if any(wl) else 0),
                     digit_products="karatsuba" if info["products"] < info["digits"] ** 2
                     else "schoolbook", unit_bounds=args.unit_bounds,
                     epilogue_warps=info["epilogue_warps"] if info["tile_ctas"] == 1 else 0)
    sampler = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ms, stage = time_plan(plan, A, C, args.steps, args.warmup, flush, stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = statistics.median(ms)
    step_ms = max_over_ranks(step_ms, ws)
    value = ws * n * n * k / (step_ms * 1e-3)
    leaf_ms = statistics.median(s["leaf_ms"] for s in stage)
    tmacs = stage[-1]["field_macs"] * info["products"]
    launches = stage[-1]["launches"]

    # roofline of the dominant kernel (the grouped tensor-core leaf launch)
    peaks, peak_src = measured_peaks()
    long_step = step_ms > 100.0
    peak = peaks["bf16_tflops_sustained" if long_step else "bf16_tflops"]
    achieved = 2.0 * tmacs / (leaf_ms * 1e-3) / 1e12
    pair = info["leaf"] == ffsyrk.LEAF_TC_BF16 and info["tile_ctas"] == 2
    kernel_file = "kern_leaf_tc2.cu" if pair else "kern_leaf_tc.cu"
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": kernel_traffic(kernel_file, args.workload,
                                          plan_signature(info, args.unit_bounds)),
                "plan": plan_signature(info, args.unit_bounds),
                "kernel": ("k_leaf_tc2 (tcgen05 kind::f16 cta_group::2, 256x256 tiles on SM pairs, "
                           "bf16 digits, fp32 TMEM)" if pair else
                           "k_leaf_tc (tcgen05 kind::f16, 128x256 tiles, bf16 digits, fp32 TMEM)"),
                "peak_source": f"{peak_src} {'sustained' if long_step else 'burst'} bf16 dense",
                "algorithmic_flops_per_launch": 2.0 * tmacs,
                "leaf_ms": leaf_ms,
                "stage_ms": {"prep": statistics.median(s["prep_ms"] for s in stage),
                             "leaf": leaf_ms,
                             "post": statistics.median(s["post_ms"] for s in stage)}}

    # bit-exactness (not timed): the whole lower triangle against the
    # oracle's stored digest where tests/golden has one, and the rows the CPU
    # baseline computes with the oracle below
    C_res = C.cpu() if rank == 0 and not args.no_check else None
    # accumulator units of the leaf: the worst-case schedule's and those it ran
    units = plan.units() if args.leaf == "tc" else None
    plan.close()
    del plan

    # comparators: classical SYRK from the same leaves; the same method on the
    # warp-level INT8 tensor leaf and on the CUDA-core int64 leaf, each with
    # its leaf's multiply-add rate against the measured rate of its pipe
    compare = {}
    if not args.no_compare:
        from paper_2001_04109_gb300.ffsyrk import probe_pipe
        pipe_peak = {"i8": probe_pipe("mma_s8s8", iters=2048, reps=3),
                     "i64": probe_pipe("mad_wide_u32", iters=512, reps=3)}
        legs = [("classical_tc", "tc", 0, None), ("fast_i8", "i8", info["levels"], None),
                ("classical_i8", "i8", 0, None), ("fast_i64", "i64", info["levels"], None),
                ("classical_i64", "i64", 0, None)]
        if any(info["winograd"]):
            # the same depth with the general products computed classically
            legs.append(("fast_tc_no_winograd", "tc", info["levels"], 0))
        if info["products"] < info["digits"] ** 2:
            # the same plan with the D² schoolbook digit products
            legs.append(("fast_tc_schoolbook_digits", "tc", info["levels"], "schoolbook"))
        for name, leaf, lv, wg in legs:
            dp = None
            if wg == "schoolbook":
                dp, wg = "schoolbook", same_opts["winograd"]
            pl = ffsyrk.Plan(p, n, k, leaf=leaf, levels=lv, winograd=wg, digit_products=dp,
                             tile_ctas=args.tile_ctas if wg == 0 else None)
            slow = leaf != "tc" and n * n * k > 2 ** 36  # calls of 0.1 s or more
            st = 2 if slow else max(3, min(args.steps, 5))
            cms, cstage = time_plan(pl, A, C, st, 1 if slow else 2, flush, stream)
            cm = statistics.median(cms)
            pinfo = pl.info()
            leg = {"value": n * n * k / (cm * 1e-3), "ms_per_step": cm,
                   "levels": pinfo["levels"], "winograd": pinfo["winograd"][: pinfo["levels"]],
                   "leaf_ms": statistics.median(s["leaf_ms"] for s in cstage)}
            if leaf in pipe_peak:
                # leaf multiply-adds of its pipe: D² byte products per field
                # multiply-add (INT8), one 32×32→64 multiply-add (int64)
                macs = cstage[-1]["tensor_macs"]
                rate = macs / (leg["leaf_ms"] * 1e-3)
                leg["leaf_pipe"] = {"macs_per_s": rate, "peak_macs_per_s": pipe_peak[leaf],
                                    "frac": rate / pipe_peak[leaf], "digits": pinfo["digits"],
                                    "peak_source": "ffsyrk_probe_pipe in this run"}
            compare[name] = leg
            pl.close()

    # end to end through the C ABI with host buffers (ffsyrk_host): every step
    # copies its input from pinned host memory, runs the product and copies
    # the result back, all inside the library call; consecutive steps go to
    # rotating plans on their own streams (one plan per call in flight), so
    # one step's copies overlap another's compute; the value is steps / (first
    # call's start .. last copy's end).  As many plans as fit the free device
    # memory (each holds its workspace and device copies of A and C), 1 to 3.
    e2e = None
    if not args.no_e2e:
        del C
        torch.cuda.empty_cache()
        ws_b, slot_b = ffsyrk.workspace_query(
            p, n, k, **{kk: v for kk, v in same_opts.items()
                        if kk not in ("unit_bounds", "epilogue_warps")})
        need = ws_b + slot_b + 4 * n * (k + 3) + 4 * n * n
        free, _ = torch.cuda.mem_get_info()
        nfly = int(max(1, min(3, (0.9 * free) // need)))
        ceiling = copy_ceiling(n, k, stream)
        A_pin = A_host.pin_memory()
        C_pins = [torch.empty((n, n), dtype=torch.int32).pin_memory() for _ in range(nfly)]
        plans = [ffsyrk.Plan(p, n, k, **same_opts)
                 for _ in range(nfly)]
        streams = [torch.cuda.Stream() for _ in range(nfly)]

        def pipelined(nsteps):
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(streams[0])
            for s_ in streams[1:]:
                s_.wait_event(t0)
            for i in range(nsteps):
                b = i % nfly
                plans[b].host(A_pin, C_pins[b], stream=streams[b])
            for s_ in streams[1:]:
                ev = torch.cuda.Event()
                ev.record(s_)
                streams[0].wait_event(ev)
            t1.record(streams[0])
            torch.cuda.synchronize()
            return t0.elapsed_time(t1)

        # the first step's input copy and the last step's output copy overlap
        # nothing: at least 30 steps, so that they weigh on a continuous
        # stream of calls as little as they do in one
        nst = max(nfly, args.steps, 30)
        pipelined(max(nfly, args.warmup))
        e_ms = pipelined(nst) / nst
        for pl_ in plans:
            pl_.sync_status()
            pl_.close()
        del plans, C_pins
        torch.cuda.empty_cache()
        e2e = {"value": ws * n * n * k / (e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": n * k * 4, "d2h_bytes_per_step": n * n * 4,
               "ms_per_step": e_ms, "steps": nst,
               "copy_ceiling": {**ceiling,
                                "bound_ms": max(step_ms, ceiling["h2d_ms"], ceiling["d2h_ms"]),
                                "what": "plain pinned cudaMemcpyAsync of one step's A (H2D) and "
                                        "n×n C (D2H); with copies overlapping compute a step "
                                        "cannot beat the largest of those and the device step"},
               "pipeline": f"ffsyrk_host (copy A in, product, copy C out) on pinned host "
                           f"buffers, {nfly} plan(s) and stream(s) in rotation: one step's "
                           "copies overlap another's product"}

    batched = None
    if not args.no_batched and args.workload == DEFAULT_WORKLOAD:
        batched = batched_leg(steps=max(3, min(args.steps, 10)), warmup=3, check=not args.no_check)

    cpu, parity = None, None
    if rank == 0:
        rows = vals = None
        if not args.no_cpu:
            cpu, rows, vals = cpu_oracle_rate(A_host.numpy().view(np.uint32), p,
                                              budget_s=args.cpu_budget, keep_rows=True)
        if C_res is not None:
            parity = {}
            if rows is not None:
                got = C_res.numpy().view(np.uint32)[rows]
                ok = all(np.array_equal(got[t, : r + 1], vals[t, : r + 1])
                         for t, r in enumerate(rows))
                parity["rows_checked"] = int(len(rows))
                parity["rows_bit_exact"] = bool(ok)
            want = golden_digest(n, k, p)
            if want is not None:
                parity["triangle_sha256_matches_oracle"] = lower_digest(C_res) == want
            parity["bit_exact"] = all(v for kk, v in parity.items() if kk != "rows_checked")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic",
                "config": {"workload": args.workload, "description": describe(desc, info),
                           "n": n, "k": k, "p": p, "levels": info["levels"],
                           "digits": info["digits"], "digit_products": info["products"],
                           "winograd": info["winograd"][: info["levels"]],
                           "leaf": {1: "tc_bf16", 2: "i64"}[info["leaf"]],
                           "tile_ctas": info["tile_ctas"],
                           "epilogue_warps": info["epilogue_warps"],
                           "unit_bounds": args.unit_bounds,
                           "leaf_units": (None if units is None else
                                          {"worst_case": units[0], "run": units[1]}),
                           "autotuned": bool(info["autotuned"]),
                           "plan_s": plan_s,
                           "y_form": "scalar" if info["y_form"] == 0 else "2x2",
                           "l2": "flushed between steps (512 MiB write)",
                           "timing": "median of the timed steps",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "e2e": e2e, "gpu_launches": launches * args.steps, "roofline": roofline,
                "cpu_baseline": cpu, "clocks": clocks, "parity": parity, "compare": compare,
                "batched": batched}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


OPS = {
    "update": "C ← α·A·Aᵀ + β·C mod p (Section 4.2, Table 4)",
    "syrkd": "C = A·Diag(d)·Aᵀ mod p, d uniform in [1, p) (Algorithm 5)",
    "syrkbd": "C = A·B·Aᵀ mod p, B block diagonal: a 2×2 block on every third column pair (Algorithm 6)",
    "herk": "C = A·Aᴴ over F_p[i]/(i² − r), A read as n × k/2 interleaved (Re, Im) pairs (Section 3.2)",
}


def run_op(args):
    """One of the operations beyond the plain product on the workload's A, timed like it.

    The value is n²k / t with k the uint32 columns of A (for the Hermitian
    product: k/2 columns over F_{p²}); the plain product of the same A on its
    own plan is timed beside it.  Parity of these operations is checked by the
    GPU tests, not here.
    """
    import numpy as np
    import torch
    import __graft_entry__
    from paper_2001_04109_gb300 import ffsyrk, inputs

    torch.cuda.set_device(0)
    __graft_entry__.build()
    n, k, p, desc = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    A = inputs.uniform_residues(n, k, p, seed=2).cuda()
    C = inputs.uniform_residues(n, n, p, seed=3).cuda()
    C2 = torch.zeros_like(C)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(7)
    d = rng.integers(1, p, size=k).astype(np.uint32)
    e = np.zeros(max(k - 1, 0), dtype=np.uint32)
    e[0::6] = rng.integers(1, p, size=e[0::6].shape[0])
    kw = dict(leaf=args.leaf, levels=args.levels, tile_ctas=args.tile_ctas, winograd=args.winograd)
    if args.op == "herk":
        r = p - 1 if p % 4 == 3 else next(x for x in range(2, p) if pow(x, (p - 1) // 2, p) == p - 1)
        plan = ffsyrk.HerkPlan(p, r, n, k // 2, **kw)
        call = lambda: plan(A[:, : 2 * (k // 2)], C, C2, stream=stream)
        extra = {"r": r}
    else:
        plan = ffsyrk.Plan(p, n, k + 1, **kw)
        extra = {}
        if args.op == "update":
            call = lambda: plan(A, C, stream=stream, alpha=31337, beta=4242)
            extra = {"alpha": 31337, "beta": 4242}
        elif args.op == "syrkd":
            call = lambda: plan.syrkd(A, d, C, stream=stream)
        else:
            call = lambda: plan.syrkbd(A, d, e, C, stream=stream)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for s_ in range(steps):
            flush.zero_()
            ev[s_][0].record(stream)
            fn()
            ev[s_][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    sampler = ClockSampler(0)
    sampler.start()
    ms = timed(call, args.steps, args.warmup)
    clocks = sampler.stop()
    plan.sync_status()
    base = ffsyrk.Plan(p, n, k, **kw)
    base_ms = timed(lambda: base(A, C2, stream=stream), args.steps, args.warmup)
    info = base.info()
    base.close()
    plan.close()
    step_ms = statistics.median(ms)
    line = {"metric": f"{args.op}: effective ops/s (n²k/t) on 1 GB300", "value": n * n * k / (step_ms * 1e-3),
            "unit": "ops/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_ms, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "op": args.op, "description": OPS[args.op],
                       "n": n, "k": k, "p": p, "levels": info["levels"],
                       "winograd": info["winograd"][: info["levels"]],
                       "l2": "flushed between steps (512 MiB write)", **extra},
            "plain_product_ms": statistics.median(base_ms), "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def batch_problem(t, shapes, p, device):
    from paper_2001_04109_gb300 import inputs
    n, k = shapes[t]
    return inputs.uniform_residues(n, k, p, seed=BATCH["seed"] * 100000 + t, device=device)


def run_batched(args):
    """One step = one ffsyrk_batched call over all 2048 problems (device-resident)."""
    import ctypes

    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2001_04109_gb300 import ffsyrk, inputs

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    __graft_entry__.build()
    p = BATCH["p"]
    count0 = args.batch_count or BATCH["count"]
    shapes = inputs.batch_shapes(count0, BATCH["lo"], BATCH["hi"], BATCH["seed"])
    count = len(shapes)
    # all problems live in one contiguous input and one contiguous output buffer
    a_off = np.cumsum([0] + [n * k for n, k in shapes])
    c_off = np.cumsum([0] + [n * n for n, _ in shapes])
    A_all = torch.empty(int(a_off[-1]), dtype=torch.int32, device="cuda")
    C_all = torch.zeros(int(c_off[-1]), dtype=torch.int32, device="cuda")
    As = [A_all[a_off[t]:a_off[t + 1]].view(n, k) for t, (n, k) in enumerate(shapes)]
    Cs = [C_all[c_off[t]:c_off[t + 1]].view(n, n) for t, (n, _) in enumerate(shapes)]
    for t in range(count):
        As[t].copy_(batch_problem(t, shapes, p, "cuda"))
    ops = float(sum(n * n * k for n, k in shapes))
    field_macs = float(sum(n * (n + 1) // 2 * k for n, k in shapes))
    I64 = ctypes.c_int64 * count
    VP = ctypes.c_void_p * count
    ns, ks = I64(*[n for n, _ in shapes]), I64(*[k for _, k in shapes])
    pas, ldas = VP(*[a.data_ptr() for a in As]), I64(*[max(1, k) for _, k in shapes])
    pcs, ldcs = VP(*[c.data_ptr() for c in Cs]), I64(*[max(1, n) for n, _ in shapes])
    lib = ffsyrk.lib()
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def call():
        rc = lib.ffsyrk_batched(0, count, ns, ks, p, pas, ldas, pcs, ldcs, sh)
        if rc != ffsyrk.SUCCESS:
            raise ffsyrk.FfsyrkError(rc, "ffsyrk_batched")

    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    host_ms = []
    for s_ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev[s_][0].record(stream)
        call()
        ev[s_][1].record(stream)
        torch.cuda.synchronize()
        host_ms.append((time.perf_counter() - t0) * 1e3)
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    step_ms = sum(ms) / len(ms)
    step_ms = max_over_ranks(step_ms, ws)
    value = ws * ops / (step_ms * 1e-3)
    info = ffsyrk.Plan(p, 8, 8, leaf="tc", levels=0).info()
    D = info["digits"]
    peaks, peak_src = measured_peaks()
    achieved = 2.0 * D * D * field_macs / (step_ms * 1e-3) / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"],
                "unit": "TFLOP/s", "frac": achieved / peaks["bf16_tflops"],
                "traffic": None,
                "kernel": "whole step (digit split + persistent grouped leaf launch)",
                "peak_source": f"{peak_src} burst bf16 dense",
                "algorithmic_flops_per_launch": 2.0 * D * D * field_macs}
    parity = None
    if not args.no_check and rank == 0:
        import oracle
        ok = True
        picks = sorted(set([0, count - 1] + list(np.linspace(1, count - 2, 6).astype(int))))
        for t in picks:
            A_h = batch_problem(t, shapes, p, "cpu")
            want = oracle.syrk(A_h.numpy(), p, "lower")
            got = np.tril(Cs[t].cpu().numpy().view(np.uint32))
            ok &= bool(np.array_equal(got, want))
        parity = {"problems_checked": len(picks), "bit_exact": ok}
    e2e = None
    if not args.no_e2e:
        A_pin = A_all.cpu().pin_memory()
        C_pin = torch.empty_like(C_all, device="cpu").pin_memory()
        evs = []
        for it in range(1 + args.steps):
            flush.zero_()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            A_all.copy_(A_pin, non_blocking=True)
            call()
            C_pin.copy_(C_all, non_blocking=True)
            b_.record(stream)
            if it > 0:
                evs.append((a_, b_))
        torch.cuda.synchronize()
        e_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        e2e = {"value": ws * ops / (e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(4 * n * k for n, k in shapes)),
               "d2h_bytes_per_step": int(sum(4 * n * n for n, _ in shapes)), "ms_per_step": e_ms}
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_batched_rate(shapes, p, args.cpu_budget)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic",
                "config": {"workload": "batched", "description": BATCH["description"],
                           "count": count, "sum_n2k": ops, "p": p, "levels": 0,
                           "leaf": "tc_bf16", "scheduling": "device work queue, graph replay",
                           "l2": "flushed between steps (512 MiB write)",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "latency_ms": {"device_per_call": step_ms, "host_call_to_done": statistics.median(host_ms)},
                "e2e": e2e, "gpu_launches": 3 * args.steps, "roofline": roofline,
                "cpu_baseline": cpu, "clocks": clocks, "parity": parity}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def batched_leg(steps, warmup, check=True):
    """The 2048-problem batch (seeded shapes, p = 65521) as one ffsyrk_batched call per step.

    Device-resident inputs, L2 flushed between steps, CUDA events on the
    launching stream; the result checked against the oracle's stored digest
    of every problem's triangle (tests/golden) when present.
    """
    import ctypes

    import numpy as np
    import torch

    from paper_2001_04109_gb300 import ffsyrk, inputs
    p = BATCH["p"]
    shapes = inputs.batch_shapes(BATCH["count"], BATCH["lo"], BATCH["hi"], BATCH["seed"])
    count = len(shapes)
    a_off = np.cumsum([0] + [n * k for n, k in shapes])
    c_off = np.cumsum([0] + [n * n for n, _ in shapes])
    A_all = torch.empty(int(a_off[-1]), dtype=torch.int32, device="cuda")
    C_all = torch.zeros(int(c_off[-1]), dtype=torch.int32, device="cuda")
    As = [A_all[a_off[t]:a_off[t + 1]].view(n, k) for t, (n, k) in enumerate(shapes)]
    Cs = [C_all[c_off[t]:c_off[t + 1]].view(n, n) for t, (n, _) in enumerate(shapes)]
    for t in range(count):
        As[t].copy_(batch_problem(t, shapes, p, "cuda"))
    I64, VP = ctypes.c_int64 * count, ctypes.c_void_p * count
    args = (0, count, I64(*[n for n, _ in shapes]), I64(*[k for _, k in shapes]), p,
            VP(*[a.data_ptr() for a in As]), I64(*[max(1, k) for _, k in shapes]),
            VP(*[c.data_ptr() for c in Cs]), I64(*[max(1, n) for n, _ in shapes]))
    lib = ffsyrk.lib()
    stream = torch.cuda.current_stream()

    def call():
        rc = lib.ffsyrk_batched(*args, stream.cuda_stream)
        if rc != ffsyrk.SUCCESS:
            raise ffsyrk.FfsyrkError(rc, "ffsyrk_batched")

    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for s_ in range(steps):
        flush.zero_()
        ev[s_][0].record(stream)
        call()
        ev[s_][1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    ops = float(sum(n * n * k for n, k in shapes))
    out = {"workload": "batched", "description": BATCH["description"], "value": ops / (ms * 1e-3),
           "unit": UNIT, "ms_per_step": ms, "steps": steps, "sum_n2k": ops,
           "scheduling": "digit split of every problem, then one persistent leaf launch over "
                         "every problem's tiles from a device work queue, replayed as a CUDA graph"}
    if check:
        want = None
        try:
            for line in open(os.path.join(ROOT, "tests", "golden", "fullsize_sha256.txt")):
                f = line.split()
                if f and f[0] == "batched" and f[1:6] == [str(BATCH[x]) for x in
                                                          ("count", "lo", "hi", "p", "seed")]:
                    want = f[6]
        except OSError:
            pass
        if want is not None:
            h = hashlib.sha256()
            C_host = C_all.cpu().numpy().view(np.uint32)
            for t, (n, _) in enumerate(shapes):
                Ct = C_host[c_off[t]:c_off[t + 1]].reshape(n, n).astype("<u4", copy=False)
                for i in range(n):
                    h.update(Ct[i, : i + 1].tobytes())
            out["triangles_sha256_match_oracle"] = h.hexdigest() == want
    del A_all, C_all, flush
    torch.cuda.empty_cache()
    return out


def cpu_batched_rate(shapes, p, budget_s):
    """The oracle on whole problems of the batch (spread over the size range) within a budget."""
    import oracle
    order = sorted(range(len(shapes)), key=lambda t: shapes[t][0] * shapes[t][0] * shapes[t][1])
    picks = order[:: max(1, len(order) // 64)]
    done_ops, t_used, used = 0.0, 0.0, 0
    for t in picks:
        n, k = shapes[t]
        A = batch_problem(t, shapes, p, "cpu").numpy()
        t0 = time.perf_counter()
        oracle.syrk(A, p, "lower")
        t_used += time.perf_counter() - t0
        done_ops += n * n * k
        used += 1
        if t_used > budget_s:
            break
    return {"value": done_ops / t_used, "unit": UNIT, "cores": oracle.default_threads(),
            "kind": "oracle", "sample": f"{used} whole problems of the batch spread over the size "
                                        f"range ({t_used:.1f} s)"}


def run_probe_pipes():
    """Measured multiply-adds per second of each pipe a leaf can use (ffsyrk_probe_pipe)."""
    import torch

    import __graft_entry__
    from paper_2001_04109_gb300 import ffsyrk
    torch.cuda.set_device(0)
    __graft_entry__.build()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sampler = ClockSampler(0)
    sampler.start()
    rates = {}
    for kind in ffsyrk.PIPES:
        iters = 2048 if kind == "mad_wide_u32" else 8192
        ffsyrk.probe_pipe(kind, iters=iters // 8, reps=1)  # warm-up
        rates[kind] = ffsyrk.probe_pipe(kind, iters=iters, blocks=4 * sms, reps=5)
    clocks = sampler.stop()
    out = {"probe": "multiply-adds per second (median of 5 launches), register operands, "
                    f"8 independent chains per thread, {4 * sms} blocks of 256 threads",
           "macs_per_s": rates, "clocks": clocks}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched"], default=DEFAULT_WORKLOAD)
    ap.add_argument("--levels", type=int, default=None)
    ap.add_argument("--winograd", type=int, default=None,
                    help="levels of Algorithm 1 for the general products (default: cost model)")
    ap.add_argument("--leaf", choices=["tc", "i64"], default="tc")
    ap.add_argument("--tile-ctas", type=int, choices=[0, 1, 2], default=0,
                    help="tensor-core leaf tiles: 0 auto, 1 one SM, 2 SM pairs")
    ap.add_argument("--digit-products", choices=["auto", "schoolbook", "karatsuba"], default="auto",
                    help="tensor-core leaf digit products (default: Karatsuba where it applies)")
    ap.add_argument("--epilogue-warps", type=int, choices=[0, 8, 16], default=0,
                    help="one-SM tensor-core leaf: epilogue warps (0 = automatic)")
    ap.add_argument("--unit-bounds", choices=["data", "worst"], default="data",
                    help="tensor-core leaf: accumulator units from the operands' digits "
                         "(default) or from the worst-case digit magnitudes")
    ap.add_argument("--no-autotune", action="store_true",
                    help="the default workload without the autotuner (depth from the cost model)")
    ap.add_argument("--autotune", action="store_true",
                    help="let the plan time its candidate variants at the workload's size "
                         "(the default for the default workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 2048-problem batch the default workload's line also reports")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--ref-budget", type=float, default=6.0)
    ap.add_argument("--batch-count", type=int, default=None,
                    help="problems in the batched workload (default 2048; fewer for profiling)")
    ap.add_argument("--op", choices=["syrk"] + sorted(OPS), default="syrk",
                    help="time another operation on the workload's A instead of the plain product")
    ap.add_argument("--shape", type=int, nargs=3, metavar=("N", "K", "P"), default=None,
                    help="replace the workload's n, k and p (for profiling other sizes)")
    ap.add_argument("--probe-pipes", action="store_true",
                    help="print the measured multiply-add rates of the arithmetic pipes and exit")
    args = ap.parse_args()
    if args.probe_pipes:
        return run_probe_pipes()
    if args.shape is not None and args.workload != "batched":
        n_, k_, p_ = args.shape
        WORKLOADS[args.workload] = (n_, k_, p_, f"A·Aᵀ mod p, A {n_}×{k_}, p={p_}")
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        # each step one bounded oracle sample; the whole run stays within a few minutes
        args.ref_budget = min(args.ref_budget, 150.0 / (args.steps + args.warmup))
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.op != "syrk":
        return run_op(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
