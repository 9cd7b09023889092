#!/usr/bin/env python3
"""Benchmark: log det evaluations per second of the Matern alpha=2 GMRF prior.

Workload (one step = one batch): the 13-point Matern precision
Q = (kappa^2 I - Lap)^2 on a 1024 x 1024 Dirichlet-truncated grid (n = 1,048,576),
probing vectors from the distance-2 greedy colouring of the graph of Q
(18 colours), N = 20 quadrature nodes, each shifted system to relative
residual 1e-6, FP32 vectors with FP64 scalars and reductions; the batch is 16
kappa^2 values drawn log-uniformly in [0.01, 1] (seeded).  Inputs are synthetic
and seeded; the CG working set (~0.45 GB) exceeds the 129 MB L2.

Lines printed (rank 0): one JSON line per run.  `--impl reference` times the
CPU oracle (banded Cholesky log det, Sec. 2's traditional method) on a bounded
leading block of the same matrix and scales to the full size.

Multi-GPU (torchrun): each rank evaluates its own seeded kappa^2 batch (weak
scaling, no data-path collective); timing is the max over ranks.
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
sys.path.insert(0, ROOT)

import synth  # noqa: E402

DIMS = (1024, 1024)
DIST = 2
NSHIFT = 20
TOL = 1e-6
BATCH = 16
SEED = 2
METRIC = "log-det(+grad) evals/sec (Matern 1024^2, probing d=2, N=20)"
UNIT = "evals/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_FLOPS_PER_VC = 25          # 13-point pass: r, p updates (4), two direct-form 5-point
                                # levels (5 each) and the scale (1), dot products (10)
FP64_PEAK_GFLOPS = 1250.0       # measured non-tensor FP64 rate of a GB300


def peak_hbm():
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            idx = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", idx, "--query-gpu=" + q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if "Active" in s[3 + k]
                          and "Not" not in s[3 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_draws(rank: int, count: int):
    """kappa^2 draws of one rank: an independent seeded batch per rank (weak scaling)."""
    return synth.kappa2_draws(SEED + 1000 * rank, count)


def colour_ranges(n_colours: int, world: int):
    """Contiguous colour ranges [a, b) splitting one evaluation over `world` ranks
    (sizes differ by at most one); partial log dets of the ranges add up."""
    base, extra = divmod(n_colours, world)
    out, a = [], 0
    for r in range(world):
        b = a + base + (1 if r < extra else 0)
        out.append((a, b))
        a = b
    return out


def algorithmic_bytes(n, T, prec, tile_iters, passes):
    """Algorithmic HBM bytes of the CG passes of a solve.

    A pass reads r, w, p of one set and writes r, w, p of the other: 6 vector passes of
    n*T words per active tile (tile_iters counts tile-passes), plus each vertex's colour
    once per pass (4 bytes).  Halo re-reads are not counted.
    """
    w = 8 if prec == "fp64" else 4
    return 6 * n * T * w * tile_iters + 4 * n * passes


def pass_kernel_sha256():
    """sha256 over the sources of the pass kernels (device code and their launcher)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("engine_device.cuh", "engine_iter.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1105_5256_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def recorded_traffic(tile_width):
    """DRAM bytes per full launch of the pass kernel from the committed ncu summary, or
    None when the engine source changed since that capture (or no summary matches)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_stream2d_matern1024_T%d.md" % tile_width)
    try:
        rec = dict(line.split(": ", 1) for line in open(path).read().splitlines()
                   if line.startswith(("engine_sha256: ", "traffic_bytes_per_launch: ")))
        cur = pass_kernel_sha256()
        if rec.get("engine_sha256", "").strip() != cur:
            return None
        return float(rec["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def run_batch(args):
    """Secondary workload: 256 independent 2D GMRFs of uneven size (sides 32..512,
    5-point d=4 or 13-point d=2, kappa^2 log-uniform) in one persistent launch per step;
    mixed precision, with the same batch in the plain FP64 form beside it."""
    import torch
    import paper_1105_5256_gb300 as L
    torch.cuda.set_device(0)
    L.library(build_if_missing=True)
    insts = synth.batch_instances(3, count=256)
    mats = [L.grid_matrix(i.kind, i.dims, i.kappa2) for i in insts]
    dists = [i.distance for i in insts]
    out = {}
    for name, prec in (("mixed", L.LD_MIXED), ("fp64", L.LD_FP64)):
        b = L.ld_batch_create(mats, dists, NSHIFT, TOL, L.options(precision=prec))
        for _ in range(args.warmup):
            L.ld_batch_logdet(b)
        ms = 0.0
        for _ in range(args.steps):
            vals, _, info = L.ld_batch_logdet(b)
            ms += info["ms"]
        out[name] = {"value": 256 * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                     "vals": vals}
        del b
    rel = float(np.max(np.abs(out["mixed"]["vals"] - out["fp64"]["vals"]) / np.abs(out["fp64"]["vals"])))
    line = {"metric": "log-det evals/sec (batch of 256 uneven 2D GMRFs, one persistent launch)",
            "value": out["mixed"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out["mixed"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 vectors / f64 scalars", "data": "synthetic (seeded batch)",
            "config": {"workload": "256 grids, sides U{32..512}, 5-pt d=4 / 13-pt d=2, N=20, tol 1e-6",
                       "points": int(sum(i.n for i in insts))},
            "fp64_form": {"value": out["fp64"]["value"], "ms_per_step": out["fp64"]["ms_per_step"],
                          "mixed_vs_fp64_rel_diff_max": rel}}
    print(json.dumps(line), flush=True)


def run_small_configs(args):
    """The other two configurations, one JSON line each:
    periodic64: Q = 0.5 I - Lap on a 64 x 64 torus (5-point) given as a CSR matrix, distance 4,
      N = 20, tol 1e-10, FP64; log det per evaluation;
    posterior2048: Q_p = 0.1 I - Lap + 4 diag(mask) on 2048 x 2048 (10 % observed, seeded),
      distance 4, N = 20, gradient (kappa^2, tau) per evaluation, mixed precision with
      reliable updates (tol 1e-9) and the plain FP64 form beside it."""
    import torch
    import paper_1105_5256_gb300 as L
    torch.cuda.set_device(0)
    L.library(build_if_missing=True)
    peak, src = peak_hbm()
    # periodic 64^2, FP64, as a general CSR matrix (kappa^2 I - Lap on the torus)
    dims, k2 = (64, 64), 0.5
    rows, cols, w = synth.torus_edges(*dims)
    rp, ci, vv = synth.csr_from_edges(dims[0] * dims[1], rows, cols, w, k2)
    ctx = L.ld_create(L.csr_matrix(rp, ci, vv), 4, 20, 1e-10,
                      L.options(precision=L.LD_FP64, lambda_min=k2, lambda_max=k2 + 8.0))
    for _ in range(args.warmup):
        L.ld_logdet(ctx)
    ms = 0.0
    for _ in range(args.steps):
        v, info = L.ld_logdet(ctx)
        ms += info["ms"]
    print(json.dumps({"metric": "log-det evals/sec (64^2 periodic 5-point as CSR, d=4, N=20, FP64)",
                      "value": args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                      "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "periodic 64x64 CSR, kappa^2 0.5, d=4, N=20, tol 1e-10",
                                 "n_colours": info["n_colours"], "iters": info["iters"],
                                 "engine": info["engine"]},
                      "logdet": v, "quad_cert": info["quad_cert"]}),
          flush=True)
    # 2048^2 Gauss-linear posterior with gradient
    dims, k2, tau = (2048, 2048), 0.1, 4.0
    n = dims[0] * dims[1]
    mask = synth.obs_mask(4, n, 0.1)
    out = {}
    for name, prec, tol, delta in (("mixed", L.LD_MIXED, 1e-9, 1e-2), ("fp64", L.LD_FP64, 1e-9, 0.0)):
        ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D5, dims, k2, tau=tau, obs_mask=mask), 4, 20, tol,
                          L.options(precision=prec, reliable_delta=delta))
        for _ in range(max(1, args.warmup // 3)):
            L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2, L.LD_P_TAU])
        ms, it_ms, tile_iters, passes = 0.0, 0.0, 0, 0
        for _ in range(args.steps):
            v, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2, L.LD_P_TAU])
            ms += info["ms"]
            it_ms += info["iter_ms"]
            tile_iters += info["tile_iters"]
            passes += info["iters"]
        out[name] = (v, g, info, ms, it_ms, tile_iters, passes)
        del ctx
    v, g, info, ms, it_ms, tile_iters, passes = out["mixed"]
    T = info["tile_width"]
    alg = 8 * n * T * 4 * tile_iters + (4 + 4) * n * passes     # r, w, p, x_lo in and out; colour, diag
    vf, gf, infof, msf = out["fp64"][:4]
    print(json.dumps({"metric": "log-det+grad evals/sec (2048^2 Gauss-linear posterior, d=4, N=20)",
                      "value": args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                      "higher_is_better": True, "dtype": "f32 vectors / f64 scalars", "data": "synthetic",
                      "config": {"workload": "2048x2048, kappa^2 0.1, tau 4, 10% mask, grad (kappa^2, tau), tol 1e-9",
                                 "n_colours": info["n_colours"], "tile_width": T, "iters": info["iters"],
                                 "reliable_updates": info["reliable_updates"],
                                 "rel_resid_max": info["rel_resid_max"]},
                      "roofline": {"bound": "hbm", "kernel": "fused CG pass (k_stream2d, 5-point)",
                                   "achieved": alg / (it_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                                   "frac": alg / (it_ms / 1e3) / 1e9 / peak, "traffic": None,
                                   "peak_source": src},
                      "fp64_form": {"value": args.steps / (msf / 1e3), "rel_resid_max": infof["rel_resid_max"],
                                    "logdet_rel_diff": abs(v - vf) / abs(vf),
                                    "grad_rel_diff": [abs(a - b) / abs(b) for a, b in zip(g, gf)]}}),
          flush=True)


def run_field3d(args):
    """Secondary workload: Dirichlet 256^3, 7-point, seeded kappa^2 field, distance-6
    colouring, N = 32, tol 1e-6, mixed precision; one evaluation = log det and its
    derivative with respect to the field's scale c (kappa^2(s) = c kappa0^2(s))."""
    import torch
    import paper_1105_5256_gb300 as L
    torch.cuda.set_device(0)
    L.library(build_if_missing=True)
    dims = (args.side, args.side, args.side)
    n = dims[0] * dims[1] * dims[2]
    field = synth.kappa2_field(5, dims)
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_3D7, dims, 1.0, kappa2_field=field), 6, 32, 1e-6,
                      L.options(precision=L.LD_MIXED, tile_width=args.tile_width))
    for _ in range(args.warmup):
        L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2])
    clocks = Clocks()
    clocks.start()
    t0 = time.perf_counter()
    dev_ms = iter_ms = 0.0
    tile_iters = passes = launches = 0
    for _ in range(args.steps):
        v, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2])
        dev_ms += info["ms"]
        iter_ms += info["iter_ms"]
        tile_iters += info["tile_iters"]
        passes += info["iters"]
        launches += info["gpu_launches"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    T = info["tile_width"]
    ntiles = (info["n_colours"] + T - 1) // T
    # per tile-pass: r, w, p read and written, x read and written (gradient mode); per
    # pass: the colour and the FP32 field, once
    alg = (8 * n * T * 4) * tile_iters + (4 + 4) * n * passes
    peak, src = peak_hbm()
    achieved = alg / (iter_ms / 1e3) / 1e9
    line = {"metric": "log-det+grad evals/sec (Dirichlet %d^3, 7-point, kappa^2 field, d=6, N=32)" % args.side,
            "value": args.steps / (dev_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 vectors / f64 scalars",
            "data": "synthetic (seeded kappa^2 field)",
            "config": {"workload": "Dirichlet %d^3, 7-point, kappa^2 field, d=6, N=32, tol 1e-6, grad c" % args.side,
                       "n": n, "n_colours": info["n_colours"], "tile_width": T,
                       "passes_per_eval": passes / args.steps},
            "clocks": clk,
            "e2e": {"value": args.steps / wall, "unit": UNIT, "h2d_bytes_per_step": 16,
                    "d2h_bytes_per_step": 16},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "kernel": "fused CG pass (k_stream3d)", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                         "algorithmic_bytes_per_launch": 8 * n * T * 4 * ntiles + 8 * n,
                         "peak_source": src},
            "logdet": v, "grad_c": float(g[0])}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_1105_5256_gb300 as L

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    L.library(build_if_missing=True)
    prec = L.LD_MIXED if args.precision == "mixed" else L.LD_FP64
    draws = rank_draws(rank, args.batch)
    if args.kappa2 > 0:
        draws = np.full(args.batch, args.kappa2)
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D13_SQ, DIMS, float(draws[0])), DIST, NSHIFT,
                      TOL, L.options(precision=prec, tile_width=args.tile_width))
    n = DIMS[0] * DIMS[1]

    def step():
        infos = []
        vals = []
        for k2 in draws:
            L.ld_set_params(ctx, float(k2))
            v, info = L.ld_logdet(ctx)
            vals.append(v)
            infos.append(info)
        return vals, infos

    for _ in range(args.warmup):
        step()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks()
    clocks.start()
    t0 = time.perf_counter()
    dev_ms = 0.0
    iter_ms = 0.0
    tile_iters = 0
    launches = 0
    all_infos = []
    vals = []
    for _ in range(args.steps):
        v, infos = step()
        vals.extend(v)
        all_infos.extend(infos)
        for i in infos:
            dev_ms += i["ms"]
            iter_ms += i["iter_ms"]
            tile_iters += i["tile_iters"]
            launches += i["gpu_launches"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    # max over ranks of device time and of wall time
    if ws > 1:
        t = torch.tensor([dev_ms, wall], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dev_ms, wall = float(t[0]), float(t[1])
    evals = args.batch * args.steps * ws
    value = evals / (dev_ms / 1e3)
    e2e = evals / wall
    info0 = all_infos[0]
    T = info0["tile_width"]
    ncols = ((info0["n_colours"] + T - 1) // T) * T
    ntiles = ncols // T
    passes = sum(i["iters"] for i in all_infos)
    alg = algorithmic_bytes(n, T, args.precision, tile_iters, passes)
    achieved = alg / (iter_ms / 1e3) / 1e9
    peak, src = peak_hbm()
    traffic = recorded_traffic(T) if args.precision == "mixed" else None
    if args.precision == "fp64":
        # FP64 issue-bound: 25 flops per vertex-column per pass against the measured
        # 1.25 TFLOP/s non-tensor FP64 rate
        flops = FP64_FLOPS_PER_VC * n * T * tile_iters
        roof = {"bound": "alu", "kernel": "fused CG pass (k_stream2d, FP64)",
                "achieved": flops / (iter_ms / 1e3) / 1e9, "peak": FP64_PEAK_GFLOPS,
                "unit": "GFLOP/s", "traffic": None,
                "peak_source": "measured FP64 FMA-chain rate (equals the nominal 1.25 TFLOP/s)"}
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        roof = None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 vectors / f64 scalars" if args.precision == "mixed" else "f64",
        "data": "synthetic (seeded kappa^2 draws; no dataset)",
        "config": {"workload": "Matern alpha=2 (kappa^2 I - Lap)^2, 1024x1024 Dirichlet, 13-point",
                   "n": n, "colouring_distance": DIST, "n_colours": info0["n_colours"],
                   "n_shifts": NSHIFT, "tol": TOL, "batch_kappa2_draws": args.batch,
                   "precision": args.precision, "tile_width": info0["tile_width"],
                   "engine": info0["engine"], "parallelism": "dp%d (independent batches)" % ws,
                   "l2": "CG working set %.2f GB (r, p, p') > 129 MB L2" % (3 * n * ncols * (4 if args.precision == "mixed" else 8) / 1e9)},
        "clocks": clk,
        "e2e": {"value": e2e, "unit": UNIT,
                "h2d_bytes_per_step": args.batch * (3 * 8 + 2 * NSHIFT * 16),
                "d2h_bytes_per_step": args.batch * (2 * 8 + 2 * 4 + 4 * ncols)},
        "gpu_launches": launches,
        "roofline": roof or {"bound": "hbm", "kernel": "fused CG pass (k_stream2d)",
                             "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "algorithmic_bytes_per_launch": algorithmic_bytes(n, T, args.precision, ntiles, 1),
                             "peak_source": src},
        "iters_mean": float(np.mean([i["iters"] for i in all_infos])),
        "logdet_first": vals[0],
    }
    if rank == 0 and ws == 1 and args.precision == "mixed" and args.fp64_sample > 0:
        out["fp64_form"] = fp64_form(L, draws[:args.fp64_sample], vals[:args.fp64_sample])
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def fp64_form(L, draws, mixed_vals):
    """The plain FP64 form on the first draws of the batch: evaluations per second and
    the largest relative difference of the mixed-precision values from it."""
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D13_SQ, DIMS, float(draws[0])), DIST, NSHIFT,
                      TOL, L.options(precision=L.LD_FP64))
    ms = 0.0
    rel = 0.0
    for k2, vm in zip(draws, mixed_vals):
        L.ld_set_params(ctx, float(k2))
        v, info = L.ld_logdet(ctx)
        ms += info["ms"]
        rel = max(rel, abs(vm - v) / abs(v))
    return {"value": len(draws) / (ms / 1e3), "unit": UNIT, "evaluations": len(draws),
            "kappa2": [float(k) for k in draws], "mixed_vs_fp64_rel_diff_max": rel}


def cpu_baseline(budget_s: float):
    """The oracle (plain single-thread C banded Cholesky, natural order) on the leading
    principal block of the same matrix; its cost is linear in the block's rows, so the
    full-size time is the measured time scaled by n / rows."""
    from oracle import matrices as om
    from oracle import method as mt
    k2 = float(synth.kappa2_draws(SEED, BATCH)[0])
    n = DIMS[0] * DIMS[1]
    rows_per_line = DIMS[0]
    lines = 4
    # grow the sample until it takes a measurable share of the budget
    while True:
        sub = (DIMS[0], lines)
        Qs = om.precision(om.KIND_2D13_SQ, sub, k2)
        t0 = time.perf_counter()
        mt.exact_logdet_band(Qs)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or lines >= DIMS[1]:
            break
        lines *= 2
    rows = rows_per_line * lines
    full_s = dt * n / rows
    return {"value": 1.0 / full_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "banded Cholesky log det of the same model on a %dx%d grid (%d rows, "
                      "band %d, cost linear in rows) in %.2f s, scaled by n/rows = %.0f"
                      % (DIMS[0], lines, rows, 2 * DIMS[0], dt, n / rows)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    per = []
    for _ in range(max(1, args.warmup)):
        cpu_baseline(args.cpu_seconds / 4)
    samples = []
    for _ in range(args.steps):
        cb = cpu_baseline(args.cpu_seconds)
        per.append(1.0 / cb["value"])
        samples.append(cb["sample"])
    value = 1.0 / statistics.mean(per)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(per) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": "Matern alpha=2 (kappa^2 I - Lap)^2, 1024x1024 Dirichlet, 13-point"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": samples[-1]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=BATCH, help="kappa^2 values per step")
    ap.add_argument("--tile-width", type=int, default=0, help="probing vectors per tile (0 = auto)")
    ap.add_argument("--workload", default="matern1024",
                    choices=["matern1024", "batch256", "field3d256", "small"])
    ap.add_argument("--side", type=int, default=256, help="field3d256 workload: grid side")
    ap.add_argument("--fp64-sample", type=int, default=2,
                    help="draws also evaluated in the plain FP64 form (mixed precision runs)")
    ap.add_argument("--kappa2", type=float, default=0.0,
                    help="fixed kappa^2 for every evaluation (profiling runs); 0 = seeded draws")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch256":
        run_batch(args)
    elif args.workload == "field3d256":
        run_field3d(args)
    elif args.workload == "small":
        run_small_configs(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
