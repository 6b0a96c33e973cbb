"""Benchmark of the D3Q19 sweep on GB300: MLUPS and fraction of the HBM roofline.

Workload (one "step" = one Sweep = ghost exchange + fused stream/collide over
every Block): a body-force channel of 256^3 cells split into 4x4x4 Blocks of
64^3 with the on-device ghost-layer exchange, periodic along x and z, resting
walls at -y/+y, BGK tau = 0.8, force 1e-6 along x, FP32 storage and arithmetic.
Synthetic input (the state starts at rest, as in the paper's runs).  The two
PDF buffers (2 x 1.4 GB) are far larger than L2, so no flush is needed.

Run:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (the path has no data
exchange between GPUs); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, B, TAU, FORCE = 256, 64, 0.8, 1e-6
BYTES_PER_LUP = {0: 19 * 4 * 2 + 1, 1: 19 * 2 * 2 + 1, 2: 19 * 2 * 2 + 1, 3: 19 * 8 * 2 + 1}
WORKLOAD = ("D3Q19 body-force channel 256^3, 4x4x4 Blocks of 64^3 with on-device ghost "
            "exchange, periodic x/z, no-slip y walls, BGK tau=0.8, F=1e-6")
METRIC = "MLUPS"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _max_over_ranks(x, ws, device):
    """The largest x over all ranks: the slowest replica sets the job's time."""
    if ws == 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _job_value(ws, cells, steps, ms_max):
    """Whole-job throughput in MLUPS: each of ws replicas updated `cells`
    cells `steps` times, the job taking ms_max milliseconds."""
    return ws * cells * steps / (ms_max * 1e-3) / 1e6


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        smax = max(r[1] for r in rows)
        loaded = [r for r in rows if r[2] > 0.3 * max(x[2] for x in rows)] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows)}


def _oracle_sample(seconds, warm_steps=0, threads=1):
    """The FP64 oracle on a bounded sample of the workload (a 64^3 channel with
    the same boundaries and physics), stepped until `seconds` have passed, on
    `threads` host threads (OpenMP over z planes when the oracle was built with
    it; the result does not depend on the thread count)."""
    import oracle

    oracle.build()
    oracle.set_threads(threads)
    n = 64
    p = oracle.Problem(dims=(n, n, n), tau=TAU, periodic=(1, 0, 1), force=(FORCE, 0, 0))
    f = oracle.zeros(p)
    if warm_steps:
        f = oracle.run(p, f, warm_steps)
    steps, t0 = 0, time.perf_counter()
    while True:
        f = oracle.step(p, f)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds and steps >= 3:
            break
    return n**3 * steps / el / 1e6, steps, el


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    n = 64
    p = oracle.Problem(dims=(n, n, n), tau=TAU, periodic=(1, 0, 1), force=(FORCE, 0, 0))
    # each step: one oracle time step of a 64^3 block of the channel; the run
    # stays within a few minutes for the default step counts
    per_step_budget = 120.0 / max(1, args.steps + args.warmup)
    f = oracle.zeros(p)
    t_one = time.perf_counter()
    f = oracle.step(p, f)
    t_one = time.perf_counter() - t_one
    cells = n**3
    if t_one > per_step_budget:
        # shrink the sample along z so the whole run stays bounded
        nz = max(1, int(n * per_step_budget / t_one))
        p = oracle.Problem(dims=(n, n, nz), tau=TAU, periodic=(1, 0, 1), force=(FORCE, 0, 0))
        f = oracle.zeros(p)
        cells = n * n * nz
    for _ in range(args.warmup):
        f = oracle.step(p, f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.step(p, f)
    el = time.perf_counter() - t0
    v = cells * args.steps / el / 1e6
    sample = f"64x64x{cells // 4096} channel block per step, FP64 C oracle, OpenMP on {cores} threads"
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
           "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_gpu(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_1007_1388_gb300 import build

    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    import paper_1007_1388_gb300 as L
    from paper_1007_1388_gb300 import workloads as W

    L.use_torch_allocator()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    n, b = args.size, args.block
    if args.batch_only:
        out = _batch_variants(args, L, W, barrier, torch)
        if rank == 0:
            print(json.dumps({"report": "batch", "batch": out}))
        return 0

    def make(storage=L.LBM_F32, coll=L.LBM_BGK, **extra):
        kw = dict(collision=coll, force=(args.force, 0, 0), storage=storage, **W.channel_bc())
        kw.update(extra)
        return L.lbm_create((n, n, n), (b, b, b), TAU, None, L.make_params(**kw))

    main_kw = {}
    if args.storage:
        main_kw["storage"] = {"f32": L.LBM_F32, "f16s": L.LBM_F16S, "bf16s": L.LBM_BF16S,
                              "f64": L.LBM_F64}[args.storage]
        if main_kw["storage"] == L.LBM_F16S:
            main_kw["storage_scale"] = 256.0
    if args.trt:
        main_kw["coll"] = L.LBM_TRT
    if args.kernel:
        main_kw["kernel"] = {"auto": 0, "register": 1, "tma": 2}[args.kernel]
    if args.streaming == "aa":
        main_kw["streaming"] = L.LBM_STREAM_AA
    ctx = make(**main_kw)
    if not args.no_autotune:
        # pick kernel, tile and register budget by timing on this GPU (outside the timed region)
        L.lbm_autotune(ctx, None)
    info = L.lbm_get_info(ctx)
    sweep_cfg = list(L.lbm_get_sweep_config(ctx))
    cells = info.cells
    stream = ctx.stream  # the torch stream the library enqueues on

    # ---- warm-up, then the timed region: K steps, per-launch events live
    L.lbm_step(ctx, args.warmup)
    L.lbm_profile_enable(ctx, True)
    L.lbm_profile_read(ctx)  # clear
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(dev) as clk:
        torch.cuda.nvtx.range_push("timed_steps")  # a range for profilers (ncu --nvtx)
        e0.record(stream)
        L.lbm_step(ctx, args.steps)
        e1.record(stream)
        barrier()
        torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    prof = L.lbm_profile_read(ctx)
    L.lbm_profile_enable(ctx, False)
    ms_max = _max_over_ranks(ms, ws, "cuda")
    value = _job_value(ws, cells, args.steps, ms_max)

    # ---- graph-replay timing of the same step (information)
    barrier()
    e0.record(stream)
    L.lbm_step(ctx, args.steps)
    e1.record(stream)
    barrier()
    graph_mlups = cells * args.steps / (e0.elapsed_time(e1) * 1e-3) / 1e6

    peak, peak_kind = _peaks()
    sweep_ms = prof.sweep_ms / max(1, prof.sweep_launches)
    xch_ms = prof.exchange_ms / max(1, prof.exchange_launches)
    st_main = main_kw.get("storage", 0)
    alg_bytes = BYTES_PER_LUP[st_main] * cells
    achieved = alg_bytes / (sweep_ms * 1e-3) / 1e9
    aa = args.streaming == "aa"
    from paper_1007_1388_gb300 import build as _build

    traffic = (_ncu_traffic("sweep_aa_f32_channel256", _build.AA_SOURCES) if aa
               else _ncu_traffic("sweep_f32_channel256"))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_kind": peak_kind,
                "kernel": ("lbm::sweep_aa_kernel" if aa
                           else "lbm::sweep_tma_kernel" if info.kernel == L.LBM_KERNEL_TMA
                           else "lbm::sweep2_kernel" if info.pair else "lbm::sweep_kernel"),
                "bytes_per_lup": BYTES_PER_LUP[st_main], "sweep_ms": sweep_ms,
                "exchange_ms": xch_ms, "exchange_pdfs": info.exchange_pdfs}

    # ---- e2e: through the C ABI with pinned host buffers, copies included
    e2e = None
    if not args.skip_e2e:
        rho_h = torch.ones(cells, dtype=torch.float32).pin_memory()
        u_h = torch.zeros(3 * cells, dtype=torch.float32).pin_memory()
        rho_o = torch.empty(cells, dtype=torch.float32).pin_memory()
        u_o = torch.empty(3 * cells, dtype=torch.float32).pin_memory()
        # one untimed pass first (the pinned buffers' first transfers are slower)
        L.lbm_init_equilibrium(ctx, rho_h, u_h)
        L.lbm_run_to_residual(ctx, 0.0, 10, args.steps)
        L.lbm_macroscopic(ctx, rho_o, u_o)
        barrier()
        t0 = time.perf_counter()
        L.lbm_init_equilibrium(ctx, rho_h, u_h)             # H2D of the initial fields
        L.lbm_run_to_residual(ctx, 0.0, 10, args.steps)     # residual D2H every 10 steps
        L.lbm_macroscopic(ctx, rho_o, u_o)                  # D2H of the final fields
        barrier()
        el = time.perf_counter() - t0
        checks = (args.steps + 9) // 10
        e2e = {"value": ws * cells * args.steps / el / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 16 * cells / args.steps,
               "d2h_bytes_per_step": (16 * cells + 8 * R_K_HOST * checks) / args.steps,
               "calls": "lbm_init_equilibrium + lbm_run_to_residual(check_every=10) + lbm_macroscopic"}
    ctx.destroy()

    # ---- storage variants and TRT on the same workload (information)
    variants = {}
    if not args.skip_variants:
        vsteps = max(50, min(args.steps, 500))
        for name, kw in [("trt_f32", dict(coll=L.LBM_TRT)),
                         ("bgk_f16s", dict(storage=L.LBM_F16S, storage_scale=256.0)),
                         ("bgk_bf16s", dict(storage=L.LBM_BF16S)),
                         ("bgk_f64", dict(storage=L.LBM_F64)),
                         # velocity inlet (moving-wall face) at -x, pressure outlet at +x
                         ("bgk_inlet_outlet_f32", dict(periodic=(0, 0, 1), face_bc=(2, 3, 1, 1, 1, 1),
                                                       wall_u=(0.01, 0, 0), force=(0, 0, 0), rho_b=1.0)),
                         # one PDF array updated in place (AA pattern)
                         ("bgk_aa_f32", dict(streaming=L.LBM_STREAM_AA)),
                         ("bgk_aa_f16s", dict(streaming=L.LBM_STREAM_AA, storage=L.LBM_F16S,
                                              storage_scale=256.0)),
                         # every link into the -y / +y walls curved (walls 0.3 / 0.7 off the rows)
                         ("bgk_curved_walls_f32", dict(curved=(0.3, 0.7)))]:
            curved = kw.pop("curved", None)
            c = make(**kw)
            if curved is not None:
                L.lbm_set_wall_distances(c, *_wall_links(L, n, curved))
            if not args.no_autotune:
                L.lbm_autotune(c, None)
            L.lbm_step(c, 5)
            L.lbm_profile_enable(c, True)
            L.lbm_profile_read(c)
            barrier()
            e0.record(c.stream)
            L.lbm_step(c, vsteps)
            e1.record(c.stream)
            barrier()
            pr = L.lbm_profile_read(c)
            st = kw.get("storage", 0)
            sw = pr.sweep_ms / max(1, pr.sweep_launches)
            variants[name] = {
                "mlups": cells * vsteps / (e0.elapsed_time(e1) * 1e-3) / 1e6,
                "sweep_gbs": BYTES_PER_LUP[st] * cells / (sw * 1e-3) / 1e9,
                "frac": BYTES_PER_LUP[st] * cells / (sw * 1e-3) / 1e9 / peak,
                "bytes_per_lup": BYTES_PER_LUP[st],
                "device_gb": L.lbm_get_info(c).device_bytes / 1e9,
                "sweep_config": list(L.lbm_get_sweep_config(c))}
            c.destroy()

    batch = None
    if not args.skip_batch:
        batch = _batch_variants(args, L, W, barrier, torch)

    log = (lambda m: print(m, file=sys.stderr, flush=True)) if rank == 0 else None
    ttr = None
    if not args.skip_ttr:
        ttr = _time_to_residual(args, L, W, torch, log)
    precision = None
    if not args.skip_precision:
        precision = _precision(L, W, torch, args.report_size, args.precision_steps, args.report_block, log)

    cpu = None
    if rank == 0 and not args.skip_cpu:
        cores = os.cpu_count() or 1
        v, steps, el = _oracle_sample(args.cpu_seconds, threads=cores)
        v1, steps1, el1 = _oracle_sample(args.cpu_seconds / 2, threads=1)
        cpu = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"64^3 block of the same channel, {steps} FP64 steps in {el:.1f} s, "
                         f"C with OpenMP over z planes on {cores} threads",
               "single_thread": {"value": v1, "cores": 1,
                                 "sample": f"{steps1} steps in {el1:.1f} s on one thread"}}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": WORKLOAD, "cells": cells, "blocks": info.blocks,
                          "tile": list(info.tile), "sweep_config": sweep_cfg,
                          "parallelism": f"replicas x{ws}",
                          "l2": "inputs larger than L2 (2 x 1.4 GB PDF buffers), no flush"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": int(prof.sweep_launches + prof.exchange_launches),
               "clocks": clk.summary(), "graph_mlups": graph_mlups, "variants": variants,
               "batch": batch, "time_to_residual": ttr, "precision": precision}
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


R_K_HOST = 8  # doubles per instance read back by one residual check

BATCH_WORKLOAD = ("256 independent D3Q19 channels, per-axis sizes uniform in [16, 96], tau uniform "
                  "in [0.55, 1.2], sphere packings (radius 2-6, porosity 0.7-0.9), seed 1234, "
                  "BGK, F=1e-5 along x, walls at -y/+y")
BATCH_FORCE = 1e-5
HANDOVER_TOL = 1e-4  # FP16 storage to this residual, then FP32 (warmstart.solve_handover)


def _batch_variants(args, L, W, barrier, torch):
    """Batched launch over 256 uneven instances (one sweep launch per step, CUDA
    graph, autotuned tiling) against the same instances as 256 separate
    contexts on concurrent streams, FP32 and shifted-FP16 storage; and the
    time to residual 1e-6 of every instance, batched against separate."""
    import numpy as np

    inst = W.batch_instances(seed=1234, n=args.batch_instances)
    dims = [d for d, _, _ in inst]
    taus = [t for _, t, _ in inst]
    flags = [f for _, _, f in inst]
    steps = args.batch_steps
    out = {"workload": BATCH_WORKLOAD, "instances": len(inst), "steps": steps}
    for name, kw in [("f32", {}), ("f16s", dict(storage=L.LBM_F16S, storage_scale=256.0))]:
        p = L.make_params(collision=L.LBM_BGK, force=(BATCH_FORCE, 0, 0), **W.channel_bc(), **kw)
        ctx = L.lbm_batch_create(dims, taus, flags, p)
        if not args.no_autotune:
            L.lbm_autotune(ctx, None)
        info = L.lbm_get_info(ctx)
        L.lbm_step(ctx, 10)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        L.lbm_step(ctx, steps)
        e1.record(ctx.stream)
        barrier()
        ms = e0.elapsed_time(e1)
        res = {"mlups": info.cells * steps / (ms * 1e-3) / 1e6,
               "mflups": info.fluid_cells * steps / (ms * 1e-3) / 1e6,
               "ms_per_step": ms / steps, "cells": info.cells, "fluid_cells": info.fluid_cells,
               "tile": list(info.tile), "sweep_ctas": info.sweep_ctas,
               "sweep_config": list(L.lbm_get_sweep_config(ctx))}
        L.lbm_profile_enable(ctx, True)
        L.lbm_profile_read(ctx)
        L.lbm_step(ctx, 20)
        pr = L.lbm_profile_read(ctx)
        L.lbm_profile_enable(ctx, False)
        sw = pr.sweep_ms / max(1, pr.sweep_launches)
        st = kw.get("storage", 0)
        res["sweep_ms"] = sw
        res["sweep_gbs"] = BYTES_PER_LUP[st] * info.cells / (sw * 1e-3) / 1e9
        res["launches_per_step"] = (pr.sweep_launches + pr.exchange_launches) / 20
        ctx.destroy()
        out[name] = res
        if name == "f32" and not args.skip_ttr and not args.batch_no_separate:
            # time to residual 1e-6 (change per step over 50-step checks) of every
            # instance from rest: one batch context against one context per instance
            tt = {"tol": 1e-6, "check_every": 50, "max_steps": 30000}
            ctx = L.lbm_batch_create(dims, taus, flags, p)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, _ = L.lbm_run_to_residual_each(ctx, 1e-6, 50, 30000, interval=True)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            ctx.destroy()
            ok = st[st >= 0]
            tt["batched"] = {"wall_s": sec, "steps_mean": float(ok.mean()) if ok.size else None,
                             "steps_max": int(ok.max()) if ok.size else None, "unconverged": int((st < 0).sum())}
            ctxs = [L.lbm_create(d, d, t, f, p) for d, t, f in inst]
            st2, sec2 = _solve_contexts(L, ctxs, 1e-6, 50, 30000)
            tt["separate_contexts"] = {"wall_s": sec2, "steps_equal": bool(np.array_equal(st, st2))}
            tt["batched_over_separate"] = sec2 / sec
            res["time_to_residual"] = tt
        if args.batch_no_separate:
            continue
        # the same instances, one context (and stream) each
        ctxs = [L.lbm_create(d, d, t, f, p) for d, t, f in inst]
        for c in ctxs:
            L.lbm_step(c, 10)
        barrier()
        t0 = time.perf_counter()
        for c in ctxs:
            L.lbm_step(c, steps)
        barrier()
        el = time.perf_counter() - t0
        res["separate_mlups"] = info.cells * steps / el / 1e6
        res["batched_over_separate"] = res["mlups"] / res["separate_mlups"]
        for c in ctxs:
            c.destroy()
    return out


PRECISION_WORKLOAD = "D3Q19 lid-driven cavity 384^3, lid 0.05 along x on +y, BGK tau=0.55, 5000 steps"


def _precision(L, W, torch, n, steps, b, log=None):
    """u and rho of FP32, shifted FP16 (scale 256 and 1) and BF16 storage
    against FP64 storage of the same lid-driven cavity after `steps` steps,
    and the MLUPS of each (autotuned, CUDA events)."""
    cases = [("f64", L.LBM_F64, 1.0), ("f32", L.LBM_F32, 1.0), ("f16s_scale256", L.LBM_F16S, 256.0),
             ("f16s_scale1", L.LBM_F16S, 1.0), ("bf16s", L.LBM_BF16S, 1.0)]
    out = {"workload": PRECISION_WORKLOAD.replace("384", str(n), 1).replace("5000", str(steps)), "block": b}
    ref = None
    for name, st, scale in cases:
        torch.cuda.empty_cache()
        p = L.make_params(wall_u=(0.05, 0, 0), storage=st, storage_scale=scale, **W.cavity_bc())
        ctx = L.lbm_create((n,) * 3, (b,) * 3, 0.55, None, p)
        L.lbm_autotune(ctx, None)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        L.lbm_step(ctx, steps)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        m, _, nonfinite = L.lbm_invariants(ctx)
        rho = torch.empty(n**3, dtype=torch.float32, device="cuda")
        u = torch.empty(3 * n**3, dtype=torch.float32, device="cuda")
        L.lbm_macroscopic_device(ctx, rho, u)
        L.lbm_synchronize(ctx)
        ctx.destroy()
        rho, u = rho.double(), u.double()
        row = {"mlups": n**3 * steps / (ms * 1e-3) / 1e6, "mass": m, "nonfinite": nonfinite}
        if ref is None:
            ref = (rho, u)
            row["u_max"] = float(u.abs().max())
        else:
            du, dr = u - ref[1], rho - ref[0]
            row.update(u_max_err=float(du.abs().max()), u_rms_err=float(du.square().mean().sqrt()),
                       rho_max_err=float(dr.abs().max()), rho_rms_err=float(dr.square().mean().sqrt()))
        out[name] = row
        if log:
            log(f"{name} {row}")
        del rho, u
    del ref
    torch.cuda.empty_cache()
    return out


def run_precision_report(args):
    """Storage precision at full size (one JSON line): see _precision."""
    import torch

    torch.cuda.set_device(0)
    from paper_1007_1388_gb300 import build

    build.build()
    import paper_1007_1388_gb300 as L
    from paper_1007_1388_gb300 import workloads as W

    L.use_torch_allocator()
    out = _precision(L, W, torch, args.report_size, args.report_steps, args.report_block,
                     log=lambda m: print(m, file=sys.stderr, flush=True))
    out["report"] = "precision"
    print(json.dumps(out))
    return 0


TTR_WORKLOAD = ("held-out sphere-packed channels 64^3 (seeds 10000.., periodic x/z, walls -y/+y, spheres of "
                "radius 2-6, porosity U[0.7, 0.9], force U[5e-7, 5e-6] along x), BGK tau=0.8; residual 1e-6 = "
                "change per step over 50-step checks, per instance")


def _solve_separate(L, W, WS, flags, forces, n, tol, every, max_steps):
    """The same channels as one context each (own stream), stepped
    interleaved: every live context takes a velocity snapshot and `every`
    steps, then each is checked.  Returns (steps per instance, seconds)."""
    ctxs = [L.lbm_create((n, n, n), (n, n, n), WS.TAU, f, L.make_params(force=(F, 0, 0), **W.channel_bc()))
            for f, F in zip(flags, forces)]
    return _solve_contexts(L, ctxs, tol, every, max_steps)


def _solve_contexts(L, ctxs, tol, every, max_steps):
    """Steps single-instance contexts (own streams) interleaved until each
    one's change per step over `every` steps is below tol; destroys them.
    Returns (steps per context, -1 where not reached; seconds)."""
    import numpy as np
    import torch

    K = len(ctxs)
    steps = np.full(K, -1, np.int64)
    live, done = list(range(K)), 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while live and done < max_steps:
        for k in live:
            L.lbm_snapshot_velocity(ctxs[k])
            L.lbm_step(ctxs[k], every)
        done += every
        nxt = []
        for k in live:
            if L.lbm_residual_vs_snapshot(ctxs[k], every) < tol:
                steps[k] = done
            else:
                nxt.append(k)
        live = nxt
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    for c in ctxs:
        c.destroy()
    return steps, sec


def _time_to_residual(args, L, W, torch, log=None):
    """Time to residual 1e-6 on held-out sphere-packed channels: FP32 from
    rest (one batch context; and one context per channel), shifted-FP16
    storage handed over to FP32 at residual 1e-4, the learned warm start
    (network trained in this run), and both combined.  Wall seconds from the
    initial state to every instance converged (host-timed, checks included);
    final velocity error against the FP32 solution from rest."""
    import numpy as np
    from paper_1007_1388_gb300 import unet, warmstart as WS

    n, K, tol, every = args.ttr_size, args.ttr_eval, 1e-6, 50
    V = n ** 3
    t0 = time.perf_counter()
    samples = W.channel_samples(list(range(args.ttr_train)) + list(range(10000, 10000 + K)), n)
    ev = samples[args.ttr_train:]
    flags = [f for f, _ in ev]
    forces = [F for _, F in ev]
    out = {"workload": TTR_WORKLOAD.replace("64^3", f"{n}^3"), "instances": K, "tol": tol, "check_every": every,
           "geometry_seconds": time.perf_counter() - t0}
    u_ref = None

    def row(steps, sec, u=None):
        ok = steps[steps >= 0]
        r = {"steps_mean": float(ok.mean()) if ok.size else None,
             "steps_median": float(np.median(ok)) if ok.size else None,
             "steps_max": int(ok.max()) if ok.size else None, "unconverged": int((steps < 0).sum()),
             "wall_s": sec}
        if u is not None:
            e = [float((u[3 * V * k:3 * V * (k + 1)] - u_ref[3 * V * k:3 * V * (k + 1)]).norm()
                       / u_ref[3 * V * k:3 * V * (k + 1)].norm()) for k in range(K)]
            r["u_rel_err_mean"], r["u_rel_err_max"] = float(np.mean(e)), float(np.max(e))
        if "f32_batched" in out:
            r["speedup_wall"] = out["f32_batched"]["wall_s"] / sec
            r["speedup_steps"] = out["f32_batched"]["steps_mean"] / r["steps_mean"] if ok.size else None
        if log:
            log(f"time to residual: {r}")
        return r

    torch.cuda.nvtx.range_push("ttr_f32_batched")  # a range for profilers (ncu --nvtx)
    ctx, st, _, sec = WS.solve(flags, forces, n, tol, every)
    torch.cuda.nvtx.range_pop()
    _, u_ref = WS.fields(ctx, K, n)
    ctx.destroy()
    out["f32_batched"] = row(st, sec)
    st, sec = _solve_separate(L, W, WS, flags, forces, n, tol, every, 20000)
    out["f32_separate_contexts"] = row(st, sec)
    ctx, st, s16, _, sec = WS.solve_handover(flags, forces, n, tol, HANDOVER_TOL, every)
    _, u = WS.fields(ctx, K, n)
    ctx.destroy()
    out["f16s_then_f32"] = row(st, sec, u)
    out["f16s_then_f32"]["steps_16bit_mean"] = float(s16.mean())
    out["f16s_then_f32"]["switch_tol"] = HANDOVER_TOL
    # the learned warm start: training set solved and network trained here
    t1 = time.perf_counter()
    train = WS.make_dataset(None, n, chunk=250, tol=tol, samples=samples[:args.ttr_train])
    net = unet.UNet(n, 4, seed=1)
    losses = WS.train(net, train, epochs=args.ttr_epochs, lr=2e-3, lr_final=2e-5)
    torch.cuda.synchronize()
    out["network"] = {"train_channels": args.ttr_train, "epochs": args.ttr_epochs,
                      "train_set_solve_seconds": train.solve_seconds,
                      "train_seconds": time.perf_counter() - t1 - train.solve_seconds,
                      "loss_last": float(np.mean(losses[-50:]))}
    solid = torch.from_numpy(np.concatenate([f.reshape(-1) for f in flags])).cuda()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    init = WS.predict(net, solid, forces, n, train.s_rho, train.s_u)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t2
    e = [float((init[1][3 * V * k:3 * V * (k + 1)] - u_ref[3 * V * k:3 * V * (k + 1)]).norm()
               / u_ref[3 * V * k:3 * V * (k + 1)].norm()) for k in range(K)]
    out["network"].update(inference_seconds=t_inf, prediction_u_rel_err_mean=float(np.mean(e)))
    ctx, st, _, sec = WS.solve(flags, forces, n, tol, every, init=init)
    _, u = WS.fields(ctx, K, n)
    ctx.destroy()
    out["warm_start_f32"] = row(st, sec + t_inf, u)
    ctx, st, s16, _, sec = WS.solve_handover(flags, forces, n, tol, HANDOVER_TOL, every, init=init)
    _, u = WS.fields(ctx, K, n)
    ctx.destroy()
    out["warm_start_f16s_then_f32"] = row(st, sec + t_inf, u)
    out["warm_start_f16s_then_f32"]["steps_16bit_mean"] = float(s16.mean())
    net.destroy()
    del train, init, u, u_ref, solid
    torch.cuda.empty_cache()
    return out


SIZES_WORKLOAD = ("D3Q19 channel (periodic x/z, no-slip walls -y/+y), BGK tau=0.8, force 1e-6 along x, FP32; "
                  "cubes 64^3 .. 512^3 split into 1, 8 and 64 Blocks")


def run_sizes_report(args):
    """Domain size and Block count (Sec. 4.1's single-GPU measurements): the
    autotuned step of a channel cube of each size, as one Block and split into
    2^3 and 4^3 Blocks, with MLUPS, the sweep's fraction of the measured HBM
    bandwidth and the exchange's share.  Prints one JSON line."""
    import torch

    torch.cuda.set_device(0)
    from paper_1007_1388_gb300 import build

    build.build()
    import paper_1007_1388_gb300 as L
    from paper_1007_1388_gb300 import workloads as W

    L.use_torch_allocator()
    peak = _peaks()[0]
    rows = []
    for n, per_axis, mode in [(n, pa, m) for n in args.sizes for m in args.size_streaming
                              for pa in args.size_splits]:
        if True:
            b = n // per_axis
            streaming = L.LBM_STREAM_AA if mode == "aa" else L.LBM_STREAM_TWO_GRID
            p = L.make_params(force=(FORCE, 0, 0), streaming=streaming, **W.channel_bc())
            torch.cuda.empty_cache()
            try:
                ctx = L.lbm_create((n,) * 3, (b,) * 3, TAU, None, p)
            except L.LBMError as e:  # a Block beyond 32-bit plane offsets, or out of memory
                rows.append({"n": n, "blocks": per_axis**3, "block": b, "streaming": mode, "refused": str(e)})
                print(rows[-1], file=sys.stderr, flush=True)
                continue
            tuned = True
            try:
                L.lbm_autotune(ctx, None)
            except L.LBMError:  # in place, tuning needs a transient copy of the state
                tuned = False
            steps = int(min(2000, max(50, 3e10 // n**3)))
            L.lbm_step(ctx, 10)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            L.lbm_step(ctx, steps)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            L.lbm_profile_enable(ctx, True)
            L.lbm_profile_read(ctx)
            L.lbm_step(ctx, 20)
            pr = L.lbm_profile_read(ctx)
            L.lbm_profile_enable(ctx, False)
            sw = pr.sweep_ms / max(1, pr.sweep_launches)
            ex = pr.exchange_ms / 20
            m, _, nonfinite = L.lbm_invariants(ctx)
            row = {"n": n, "blocks": per_axis**3, "block": b, "streaming": mode, "autotuned": tuned,
                   "device_gb": L.lbm_get_info(ctx).device_bytes / 1e9, "steps": steps,
                   "mlups": n**3 * steps / (ms * 1e-3) / 1e6,
                   "sweep_hbm_frac": BYTES_PER_LUP[0] * n**3 / (sw * 1e-3) / 1e9 / peak,
                   "exchange_share": ex / (ex + sw), "sweep_config": list(L.lbm_get_sweep_config(ctx)),
                   "nonfinite": nonfinite}
            ctx.destroy()
            rows.append(row)
            print(row, file=sys.stderr, flush=True)
    print(json.dumps({"report": "sizes", "workload": SIZES_WORKLOAD, "peak_hbm_gbs": peak, "rows": rows}))
    return 0


POROUS_WORKLOAD = ("D3Q19 channel through overlapping solid spheres (radii 2-6, periodic x/z, no-slip "
                   "walls -y/+y), BGK tau=0.8, force 1e-6 along x, FP32; Block layout (64^3 Blocks) vs "
                   "the fluid-cell list layout at each porosity")


def run_porous_report(args):
    """Block layout against the fluid-cell list layout on porous media of
    several porosities: MFLUPS (fluid-cell updates per second), the sweep's
    algorithmic bytes over its time against the measured HBM peak (153 B per
    cell for Blocks, 224 B per fluid cell for the list), device memory.
    Prints one JSON line."""
    import numpy as np
    import torch

    torch.cuda.set_device(0)
    from paper_1007_1388_gb300 import build

    build.build()
    import paper_1007_1388_gb300 as L
    from paper_1007_1388_gb300 import workloads as W

    L.use_torch_allocator()
    peak = _peaks()[0]
    n = args.porous_size
    rows = []
    for phi in args.porosities:
        flags = W.overlapping_spheres(np.random.default_rng(4321), (n, n, n), phi)
        nfl = int((flags == 0).sum())
        for layout, name, bpu in ((L.LBM_LAYOUT_BLOCKS, "blocks", 153), (L.LBM_LAYOUT_SPARSE, "list", 224)):
            torch.cuda.empty_cache()
            p = L.make_params(force=(FORCE, 0, 0), layout=layout, **W.channel_bc())
            ctx = L.lbm_create((n,) * 3, (64,) * 3, TAU, flags, p)
            L.lbm_autotune(ctx, None)
            steps = int(min(1000, max(50, 2e10 // n**3)))
            L.lbm_step(ctx, 10)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            L.lbm_step(ctx, steps)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            L.lbm_profile_enable(ctx, True)
            L.lbm_profile_read(ctx)
            L.lbm_step(ctx, 20)
            pr = L.lbm_profile_read(ctx)
            L.lbm_profile_enable(ctx, False)
            sw = pr.sweep_ms / max(1, pr.sweep_launches)
            units = n**3 if layout == L.LBM_LAYOUT_BLOCKS else nfl
            row = {"porosity": nfl / n**3, "layout": name, "steps": steps,
                   "mflups": nfl * steps / (ms * 1e-3) / 1e6, "mlups": n**3 * steps / (ms * 1e-3) / 1e6,
                   "sweep_ms": sw, "bytes_per_unit": bpu,
                   "sweep_hbm_frac": bpu * units / (sw * 1e-3) / 1e9 / peak,
                   "device_gb": L.lbm_get_info(ctx).device_bytes / 1e9,
                   "sweep_config": list(L.lbm_get_sweep_config(ctx))}
            ctx.destroy()
            rows.append(row)
            print(row, file=sys.stderr, flush=True)
    print(json.dumps({"report": "porous", "workload": POROUS_WORKLOAD, "n": n, "peak_hbm_gbs": peak,
                      "rows": rows}))
    return 0


WARMSTART_WORKLOAD = ("learned warm start: 64^3 channels (periodic x/z, walls -y/+y), sphere packings "
                      "(radius 2-6, porosity U[0.7, 0.9]), force U[5e-7, 5e-6] along x, BGK tau=0.8; "
                      "training seeds 0..N-1, held-out seeds 10000..; residual 1e-6 (change per step over "
                      "50-step intervals)")


def run_warmstart_report(args):
    """The learned warm start end to end: solve the training channels, train
    the U-Net, then solve the held-out channels from rest, from the predicted
    equilibrium and from a consistent start at the predicted velocity.
    Prints one JSON line (steps, wall times, errors)."""
    import numpy as np
    import torch

    torch.cuda.set_device(0)
    from paper_1007_1388_gb300 import build

    build.build()
    import paper_1007_1388_gb300 as L
    from paper_1007_1388_gb300 import unet, warmstart as WS, workloads as W

    L.use_torch_allocator()
    n, tol, nb = args.ws_size, 1e-6, 4
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
    t0 = time.perf_counter()
    seeds = list(range(args.ws_train)) + list(range(10000, 10000 + args.ws_eval))
    samples = W.channel_samples(seeds, n)
    t_gen = time.perf_counter() - t0
    log(f"geometries: {len(samples)} in {t_gen:.1f} s")
    train = WS.make_dataset(None, n, chunk=args.ws_chunk, tol=tol, samples=samples[:args.ws_train])
    log(f"training set solved: {train.solve_seconds:.1f} s, steps mean {train.steps.mean():.0f}, "
        f"unconverged {int((train.steps < 0).sum())}")
    net = unet.UNet(n, nb, seed=1)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = WS.train(net, train, epochs=args.ws_epochs, lr=2e-3, lr_final=2e-5, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    ev = samples[args.ws_train:]
    flags = [f for f, _ in ev]
    forces = [F for _, F in ev]
    K, V = len(ev), n ** 3
    out = {"report": "warmstart", "workload": WARMSTART_WORKLOAD, "n": n, "train": args.ws_train,
           "eval": K, "epochs": args.ws_epochs, "batch": nb, "train_seconds": t_train,
           "train_steps": len(losses), "ms_per_train_step": 1e3 * t_train / max(1, len(losses)),
           "loss_first": losses[0], "loss_last": float(np.mean(losses[-50:])), "s_u": train.s_u,
           "training_set": {"solve_seconds": train.solve_seconds, "steps_mean": float(train.steps.mean())}}
    ctx_r, steps_r, _, sec_r = WS.solve(flags, forces, n, tol)
    rho_r, u_r = WS.fields(ctx_r, K, n)
    ctx_r.destroy()

    def errs(u):
        e = [float((u[3 * V * k:3 * V * (k + 1)] - u_r[3 * V * k:3 * V * (k + 1)]).norm()
                   / u_r[3 * V * k:3 * V * (k + 1)].norm()) for k in range(K)]
        return float(np.mean(e)), float(np.median(e)), float(np.max(e))

    def stats(steps, sec):
        ok = steps[steps >= 0]
        return {"steps_mean": float(ok.mean()) if ok.size else None,
                "steps_median": float(np.median(ok)) if ok.size else None,
                "unconverged": int((steps < 0).sum()), "wall_seconds": sec}

    out["from_rest"] = stats(steps_r, sec_r)
    solid = torch.from_numpy(np.concatenate([f.reshape(-1) for f in flags])).cuda()
    for smooth in (0, 1):
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        init = WS.predict(net, solid, forces, n, train.s_rho, train.s_u, smooth=smooth)
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t2
        pe = errs(init[1])
        for name, m in (("equilibrium", 0), ("consistent", 10)):
            ctx, st, _, sec = WS.solve(flags, forces, n, tol, init=init, consistent=m)
            _, u_w = WS.fields(ctx, K, n)
            ctx.destroy()
            row = stats(st, sec + t_inf)
            row.update(inference_seconds=t_inf, prediction_error_mean=pe[0], prediction_error_median=pe[1],
                       prediction_error_max=pe[2], final_error_max=errs(u_w)[2])
            row["speedup_steps"] = (out["from_rest"]["steps_mean"] / row["steps_mean"]
                                    if row["steps_mean"] else None)
            row["speedup_wall"] = sec_r / (sec + t_inf)
            out[f"warm_{name}_smooth{smooth}"] = row
            log(f"{name} smooth {smooth}: {row}")
    net.destroy()
    print(json.dumps(out))
    return 0


def _peak_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured"
    except Exception:
        return 1900.0, 1700.0, "fallback"


def run_unet_report(args):
    """Tensor-core U-Net at 64^3 x 4 samples: training-step time, and each
    convolution shape's forward and weight-gradient launch with CUDA events,
    as TFLOP/s against the measured bf16 peak.  One JSON line."""
    import numpy as np
    import torch

    torch.cuda.set_device(0)
    from paper_1007_1388_gb300 import build

    build.build()
    import paper_1007_1388_gb300 as L
    from paper_1007_1388_gb300 import unet, workloads as W

    L.use_torch_allocator()
    n, nb = args.ws_size, 4
    V = nb * n ** 3
    rng = np.random.default_rng(0)
    solid = torch.from_numpy(np.concatenate([W.channel_sample(s, n)[0].reshape(-1) for s in range(nb)])).cuda()
    target = torch.randn(V * 4, device="cuda") * 0.5
    net = unet.UNet(n, nb, seed=3)
    force = [0.5] * nb
    for _ in range(3):
        net.train_step(solid, force, target, 1e-4)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = args.unet_steps
    e0.record(net.stream)
    for _ in range(steps):
        net.train_step(solid, force, target, 1e-4)
    e1.record(net.stream)
    torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / steps
    out = torch.empty(V * 4, device="cuda")
    e0.record(net.stream)
    for _ in range(steps):
        net.predict(solid, force, out)
    e1.record(net.stream)
    torch.cuda.synchronize()
    ms_pred = e0.elapsed_time(e1) / steps
    # forward FLOPs (2 per multiply-add) of the ten convolutions and the head
    l = int(round(np.log2(n)))
    convs = [("W1a", 2, 16, 0), ("W1b", 16, 16, 0), ("W2a", 16, 32, 1), ("W2b", 32, 32, 1), ("W3a", 32, 64, 2),
             ("W3b", 64, 64, 2), ("W4a", 96, 32, 1), ("W4b", 32, 32, 1), ("W5a", 48, 16, 0), ("W5b", 16, 16, 0)]
    fwd_flops = sum(2.0 * 27 * ci * co * (nb << (3 * (l - lev))) for _, ci, co, lev in convs) + 2.0 * 16 * 4 * V
    train_flops = 3.0 * fwd_flops  # forward, backward-data and weight gradient
    peak, peak_sus, kind = _peak_bf16()
    res = {"report": "unet", "workload": f"U-Net, {nb} samples of {n}^3 (bf16 operands, FP32 accumulation, "
                                         "tcgen05 with bulk-copied planar operand slabs)",
           "ms_per_train_step": ms_step, "ms_per_prediction": ms_pred,
           "forward_gflop": fwd_flops / 1e9, "train_tflops_effective": train_flops / ms_step / 1e9,
           "forward_tflops_effective": fwd_flops / ms_pred / 1e9,
           "peak_bf16_tflops": peak, "peak_kind": kind,
           # the whole forward pass (convolutions plus the element-wise kernels between them) against
           # the tensor peak: a lower bound for the convolution kernels themselves
           "roofline": {"kernel": "lbm::conv3_bulk_kernel (whole forward pass)", "bound": "tensor",
                        "achieved": fwd_flops / ms_pred / 1e9, "peak": peak, "unit": "TFLOP/s",
                        "frac": fwd_flops / ms_pred / 1e9 / peak}}
    net.destroy()
    print(json.dumps(res))
    return 0


def _wall_links(L, n, q):
    """(cells, directions, distances) of every pull from the -y / +y walls of
    an n^3 channel: the bottom wall q[0] below row 0, the top q[1] above row n-1."""
    import numpy as np

    e = L.lbm_directions()[0]
    x, z = np.meshgrid(np.arange(n), np.arange(n))
    cells, dirs, qs = [], [], []
    for i in range(1, len(e)):
        ey = int(e[i][1])
        if ey == 0:
            continue
        y = 0 if ey == 1 else n - 1
        cells.append((x + n * (y + n * z)).ravel())
        dirs.append(np.full(n * n, i))
        qs.append(np.full(n * n, q[0] if ey == 1 else q[1]))
    return np.concatenate(cells), np.concatenate(dirs), np.concatenate(qs)


def _ncu_traffic(name, sources=None):
    """DRAM bytes per launch from the committed ncu summary, if it is current."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d[name]
        from paper_1007_1388_gb300 import build

        if ent.get("kernel_hash") != build.kernel_hash(*([sources] if sources else [])):
            return None
        return ent["dram_bytes_per_launch_full"]
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-variants", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-ttr", action="store_true", help="skip the time-to-residual block")
    ap.add_argument("--skip-precision", action="store_true", help="skip the storage-precision block")
    ap.add_argument("--precision-steps", type=int, default=2000,
                    help="steps of the precision block in the default run (--report precision: --report-steps)")
    ap.add_argument("--ttr-size", type=int, default=64)
    ap.add_argument("--ttr-eval", type=int, default=48, help="held-out channels of the time-to-residual block")
    ap.add_argument("--ttr-train", type=int, default=1000, help="training channels of its warm start")
    ap.add_argument("--ttr-epochs", type=int, default=30)
    ap.add_argument("--report", default="", choices=["", "precision", "warmstart", "unet", "sizes", "porous"],
                    help="precision: storage-precision report on the 384^3 cavity; warmstart: the learned "
                         "warm start end to end (one JSON line each)")
    ap.add_argument("--ws-size", type=int, default=64)
    ap.add_argument("--ws-train", type=int, default=2000)
    ap.add_argument("--ws-eval", type=int, default=200)
    ap.add_argument("--ws-epochs", type=int, default=40)
    ap.add_argument("--ws-chunk", type=int, default=250)
    ap.add_argument("--unet-steps", type=int, default=20)
    ap.add_argument("--report-size", type=int, default=384)
    ap.add_argument("--sizes", type=int, nargs="+", default=[64, 128, 256, 384, 512],
                    help="cube sizes of --report sizes (each divisible by 4)")
    ap.add_argument("--report-steps", type=int, default=5000)
    ap.add_argument("--report-block", type=int, default=128)
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--batch-only", action="store_true", help="only the batched workload (one JSON line)")
    ap.add_argument("--batch-no-separate", action="store_true",
                    help="skip the one-context-per-instance comparison")
    ap.add_argument("--size", type=int, default=N, help="cells per axis (profiling runs use less)")
    ap.add_argument("--block", type=int, default=B, help="cells per Block along each axis")
    ap.add_argument("--storage", default="", help="f32 | f16s | bf16s | f64 (default f32)")
    ap.add_argument("--trt", action="store_true", help="TRT instead of BGK")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default sweep configuration")
    ap.add_argument("--kernel", default="", help="auto | register | tma")
    ap.add_argument("--streaming", default="two", choices=["two", "aa"],
                    help="two PDF arrays (default) or one updated in place")
    ap.add_argument("--size-streaming", nargs="+", default=["two"], choices=["two", "aa"],
                    help="--report sizes: streaming modes to run")
    ap.add_argument("--size-splits", type=int, nargs="+", default=[1, 2, 4],
                    help="--report sizes: Blocks per axis")
    ap.add_argument("--porosities", type=float, nargs="+", default=[0.3, 0.5, 0.7, 0.9],
                    help="--report porous: fluid fractions")
    ap.add_argument("--porous-size", type=int, default=256, help="--report porous: cells per axis")
    ap.add_argument("--force", type=float, default=FORCE, help="body force along x")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.report == "precision":
        return run_precision_report(args)
    if args.report == "warmstart":
        return run_warmstart_report(args)
    if args.report == "unet":
        return run_unet_report(args)
    if args.report == "sizes":
        return run_sizes_report(args)
    if args.report == "porous":
        return run_porous_report(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
