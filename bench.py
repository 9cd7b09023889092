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

# concurrent tile groups and batch instances each need a hardware queue of their own; the
# CUDA runtime's default of 8 makes streams beyond the eighth wait on one another (read when
# the CUDA context is created, so set before torch touches the device)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

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


def algorithmic_bytes(n, T, word, tile_iters, keep_x=False, bq_per_pass=0, passes=0):
    """Algorithmic HBM bytes of the CG passes of a solve.

    A pass reads the CG state of every vertex and probing vector once and writes it
    once: r and p (4 words), plus x in gradient mode (2 words); the matrix adds its own
    bytes once per pass (0 for a constant-coefficient stencil, one word a vertex for a
    kappa^2 field, one byte a vertex for an observation mask).  tile_iters counts
    tile-passes of T columns each.
    """
    return (4 + (2 if keep_x else 0)) * n * T * word * tile_iters + bq_per_pass * passes


def moved_bytes(n, T, word, tile_iters, pass_words, lean):
    """Bytes the pass kernel moves (halo re-reads aside): its state words per vertex and
    column (ld_info.pass_words: 4 for the lean pass, 6 for the stored-w pass, 2 more with
    x) and per vertex the tile's lane code (1 byte, lean pass) or colour (4 bytes)."""
    return (pass_words * T * word + (1 if lean else 4)) * n * tile_iters


def pass_kernel_sha256(names=("engine_device.cuh", "engine_lean.cuh")):
    """sha256 over the device sources of a pass kernel (the lean lattice pass by default)."""
    import hashlib
    h = hashlib.sha256()
    for name in names:
        h.update(open(os.path.join(ROOT, "paper_1105_5256_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def recorded_traffic(profile, key="traffic_bytes_per_pass"):
    """DRAM bytes (read + write) of one CG pass (or, key traffic_bytes_per_vertex_tile_pass,
    of one vertex and tile of a pass) from a committed ncu summary under profiles/, or None
    when the pass kernel's sources changed since that capture (or the summary is missing)."""
    path = os.path.join(ROOT, "profiles", profile)
    try:
        rec = dict(line.split(": ", 1) for line in open(path).read().splitlines()
                   if line.startswith(("engine_sha256: ", "engine_sources: ", key + ": ")))
        names = tuple(rec.get("engine_sources", "engine_device.cuh engine_lean.cuh").split())
        if rec.get("engine_sha256", "").strip() != pass_kernel_sha256(names):
            return None
        return float(rec[key])
    except (OSError, KeyError, ValueError):
        return None


def combine_partials(vec):
    """Sum one evaluation's per-rank partial results (log det, then gradient components)
    over the ranks: the one exchange of the colour split (Sec. 2.1, one probing vector per
    node), a single all-reduce of 1 + n_params doubles."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(vec, dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.cpu()]


def timed_evals(L, ctx, count, params=None, grad=None):
    """Evaluate `count` times (optionally setting kappa^2 etc. first); returns the device
    time (ms), the time inside the CG passes (ms), tile-passes, passes and the last info."""
    ms = it_ms = 0.0
    tile_iters = passes = 0
    info = v = g = None
    for k in range(count):
        if params is not None:
            L.ld_set_params(ctx, *params[k % len(params)])
        if grad:
            v, g, info = L.ld_logdet_grad(ctx, grad)
        else:
            v, info = L.ld_logdet(ctx)
        ms += info["ms"]
        it_ms += info["iter_ms"]
        tile_iters += info["tile_iters"]
        passes += info["iters"]
    return dict(ms=ms, iter_ms=it_ms, tile_iters=tile_iters, passes=passes, info=info, logdet=v, grad=g)


def roofline_entry(kernel, n, T, word, r, keep_x, bq_per_pass, peak, src, traffic=None):
    alg = algorithmic_bytes(n, T, word, r["tile_iters"], keep_x, bq_per_pass, r["passes"])
    info = r["info"]
    lean = info["pass_words"] == 4 + (2 if keep_x else 0)     # the lean pass moves the algorithmic words
    achieved = alg / (r["iter_ms"] / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "algorithmic_bytes_per_pass": alg / max(r["passes"], 1),
            "moved_bytes_per_pass": moved_bytes(n, T, word, r["tile_iters"], info["pass_words"], lean)
            / max(r["passes"], 1),
            "pass_words": info["pass_words"], "peak_source": src}


def config_posterior2048(L, steps, peak, src, warmup=1, fp64=True):
    """The Gauss-linear posterior workload: Q_p = 0.1 I - Lap + 4 diag(mask) on 2048 x 2048
    (10 % observed, seeded), distance 4, N = 20, log det and gradient (kappa^2, tau) per
    evaluation; mixed precision with reliable updates (tol 1e-9) against the plain FP64
    form on the same problem."""
    dims, k2, tau = (2048, 2048), 0.1, 4.0
    n = dims[0] * dims[1]
    mask = synth.obs_mask(4, n, 0.1)
    out = {}
    for name, prec, delta in (("mixed", L.LD_MIXED, 1e-2), ("fp64", L.LD_FP64, 0.0)):
        if name == "fp64" and not fp64:
            continue
        ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D5, dims, k2, tau=tau, obs_mask=mask), 4, 20, 1e-9,
                          L.options(precision=prec, reliable_delta=delta))
        if warmup:
            timed_evals(L, ctx, warmup, grad=[L.LD_P_KAPPA2, L.LD_P_TAU])
        out[name] = timed_evals(L, ctx, steps if name == "mixed" else 1, grad=[L.LD_P_KAPPA2, L.LD_P_TAU])
        del ctx
    m = out["mixed"]
    info = m["info"]
    T = info["tile_width"]
    lean = info["pass_words"] == 6
    roof = roofline_entry("k_lean2d (5-point, seed solution kept)" if lean else "k_stream2d (5-point, stored w)",
                          n, T, 4, m, True, n, peak, src,
                          traffic=recorded_traffic("k_lean2d_posterior2048_T2.md") if lean and T == 2 else None)
    res = {"workload": "2048x2048 posterior, kappa^2 0.1, tau 4, 10% mask, d=4, N=20, tol 1e-9, grad (kappa^2, tau)",
           "value": steps / (m["ms"] / 1e3), "unit": UNIT, "evaluations": steps,
           "dtype": "f32 vectors / f64 scalars, reliable updates", "roofline": roof,
           "n_colours": info["n_colours"], "iters": info["iters"], "reliable_updates": info["reliable_updates"],
           "rel_resid_max": info["rel_resid_max"]}
    if fp64:
        f = out["fp64"]
        res["fp64_form"] = {"value": 1.0 / (f["ms"] / 1e3),
                            "logdet_rel_diff": abs(m["logdet"] - f["logdet"]) / abs(f["logdet"]),
                            "grad_rel_diff": [abs(a - b) / abs(b) for a, b in zip(m["grad"], f["grad"])]}
    return res


def config_periodic64(L, steps):
    """The small CSR workload: Q = 0.5 I - Lap on the 64 x 64 torus given as a CSR matrix, distance 4,
    N = 20, tol 1e-10, FP64 (the one-CTA-per-tile engine: L2-resident, latency-bound)."""
    dims, k2 = (64, 64), 0.5
    rows, cols, w = synth.torus_edges(*dims)
    rp, ci, vv = synth.csr_from_edges(dims[0] * dims[1], rows, cols, w, k2)
    ctx = L.ld_create(L.csr_matrix(rp, ci, vv), 4, 20, 1e-10,
                      L.options(precision=L.LD_FP64, lambda_min=k2, lambda_max=k2 + 8.0))
    timed_evals(L, ctx, 2)
    r = timed_evals(L, ctx, steps)
    info = r["info"]
    return {"workload": "periodic 64x64 as CSR, kappa^2 0.5, d=4, N=20, tol 1e-10",
            "value": steps / (r["ms"] / 1e3), "unit": UNIT, "evaluations": steps, "dtype": "f64",
            "n_colours": info["n_colours"], "iters": info["iters"], "engine": info["engine"],
            "logdet": r["logdet"], "quad_cert": info["quad_cert"],
            "roofline": {"bound": "latency", "note": "the 4096-vertex problem is L2-resident; one CTA per tile"}}


def config_field3d(L, side, steps, peak, src, fp64=True, T=0):
    """The 3D field workload: Dirichlet side^3, 7-point, seeded kappa^2 field (log kappa^2 = -2 +
    smoothed N(0,1)), distance 6, N = 32, tol 1e-6, mixed precision; one evaluation = log
    det and its derivative with respect to the field's scale c (kappa^2 = c kappa0^2)."""
    dims = (side, side, side)
    n = side ** 3
    field = synth.kappa2_field(5, dims)
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_3D7, dims, 1.0, kappa2_field=field), 6, 32, 1e-6,
                      L.options(precision=L.LD_MIXED, tile_width=T))
    timed_evals(L, ctx, 1, grad=[L.LD_P_KAPPA2])
    r = timed_evals(L, ctx, steps, grad=[L.LD_P_KAPPA2])
    info = r["info"]
    T = info["tile_width"]
    lean = r["info"]["pass_words"] == 6
    traffic = None
    if lean and T == 4:   # the 96^3 capture's bytes per vertex and tile, over this run's tile-passes
        per = recorded_traffic("k_lean3d_field96_T4.md", "traffic_bytes_per_vertex_tile_pass")
        traffic = per * n * r["tile_iters"] / max(r["passes"], 1) if per else None
    roof = roofline_entry("k_lean3d (7-point, lean, seed solution kept)" if lean else
                          "k_stream3d (7-point, stored w, seed solution kept)", n, T, 4, r, True, 4 * n, peak, src,
                          traffic=traffic)
    out = {"workload": "Dirichlet %d^3, 7-point, kappa^2 field, d=6, N=32, tol 1e-6, grad c" % side,
           "value": steps / (r["ms"] / 1e3), "unit": UNIT, "evaluations": steps,
           "dtype": "f32 vectors / f64 scalars", "n_colours": info["n_colours"], "tile_width": T,
           "passes_per_eval": r["passes"] / steps, "roofline": roof, "logdet": r["logdet"],
           "grad_c": float(r["grad"][0])}
    del ctx
    if fp64:
        c2 = L.ld_create(L.grid_matrix(L.LD_STENCIL_3D7, dims, 1.0, kappa2_field=field), 6, 32, 1e-6,
                         L.options(precision=L.LD_FP64))
        f = timed_evals(L, c2, 1, grad=[L.LD_P_KAPPA2])
        out["fp64_form"] = {"value": 1.0 / (f["ms"] / 1e3),
                            "logdet_rel_diff": abs(r["logdet"] - f["logdet"]) / abs(f["logdet"]),
                            "grad_rel_diff": abs(float(r["grad"][0]) - float(f["grad"][0])) / abs(float(f["grad"][0]))}
    return out


def mesh_problem(side, k2h2=0.1, alpha=2):
    """Seeded perturbed side x side-vertex triangulation of the unit square with its P1 FEM
    SPDE precision (Sec. 3's SPDE model on a general mesh): kappa^2 = k2h2 / h^2 so that
    kappa^2 h^2 matches a lattice kappa^2 of k2h2.  The spectral interval is a bound from
    the lumped mass c (one third of each incident triangle's area): lambda_min >=
    kappa^4 min(c)^2 / max(c) for alpha = 2 (kappa^2 min(c) for alpha = 1), lambda_max <=
    the largest absolute row sum."""
    from paper_1105_5256_gb300 import mesh
    p, t = synth.perturbed_triangulation(6, side, side)
    h = 1.0 / (side - 1)
    k2 = k2h2 / h ** 2
    rp, ci, vv = mesh.spde_csr(p, t, k2, alpha, 1.0)
    e1, e2 = p[t[:, 1]] - p[t[:, 0]], p[t[:, 2]] - p[t[:, 0]]
    area = 0.5 * np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    c = np.bincount(t.ravel(), weights=np.repeat(area / 3.0, 3), minlength=p.shape[0])
    lo = k2 * k2 * c.min() ** 2 / c.max() if alpha == 2 else k2 * c.min()
    hi = float(np.add.reduceat(np.abs(vv), rp[:-1]).max())
    return rp, ci, vv, lo, hi


def config_mesh(L, side, steps, peak, src, matfree=True, fp64=True, T=0):
    """General-mesh input: the alpha = 2 FEM SPDE precision on a perturbed side x side-vertex
    triangulation as a CSR matrix, distance 2 in G(Q), N = 20, tol 1e-6; mixed precision on
    the fused CSR pass, beside the plain FP64 form and the matrix-free path with a cuSPARSE
    CSR product (torch) as the caller's callback, both FP64."""
    import torch
    rp, ci, vv, lo, hi = mesh_problem(side)
    n, nnz = rp.size - 1, ci.size
    out = {}
    for name, prec in (("mixed", L.LD_MIXED), ("fp64", L.LD_FP64)):
        if name == "fp64" and not (fp64 or matfree):
            continue
        ctx = L.ld_create(L.csr_matrix(rp, ci, vv), 2, 20, 1e-6,
                          L.options(precision=prec, lambda_min=lo, lambda_max=hi,
                                    tile_width=T if name == "mixed" else 0))
        timed_evals(L, ctx, 1)
        out[name] = timed_evals(L, ctx, steps if name == "mixed" else 1)
        col, nc = L.ld_get_colouring(ctx)
        del ctx
    m, f = out["mixed"], out.get("fp64")
    info = m["info"]
    T = info["tile_width"]
    # the matrix once per pass: nnz (4-byte index + 4-byte value) + the 8-byte row pointer
    traffic = None
    if T == 4:   # the 512^2 capture's bytes per vertex and tile, over this run's tile-passes
        per = recorded_traffic("k_csr_spmv_mesh512_T4.md", "traffic_bytes_per_vertex_tile_pass")
        traffic = per * n * m["tile_iters"] / max(m["passes"], 1) if per else None
    roof = roofline_entry("k_csr_step + k_csr_spmv (CSR)", n, T, 4, m, False, nnz * 8 + 8 * n, peak, src,
                          traffic=traffic)
    res = {"workload": "perturbed %dx%d-vertex triangulation, P1 FEM SPDE alpha=2, kappa^2 h^2 0.1, "
                       "d=2, N=20, tol 1e-6" % (side, side),
           "value": steps / (m["ms"] / 1e3), "unit": UNIT, "evaluations": steps,
           "dtype": "f32 vectors / f64 scalars", "n": n, "nnz": nnz, "n_colours": info["n_colours"],
           "tile_width": T, "iters": info["iters"], "engine": info["engine"], "roofline": roof,
           "lambda_bounds": [lo, hi]}
    if f is not None:
        res["fp64_form"] = {"value": 1.0 / (f["ms"] / 1e3), "iters": f["info"]["iters"],
                            "logdet_rel_diff": abs(m["logdet"] - f["logdet"]) / abs(f["logdet"])}
    if matfree:
        Qt = torch.sparse_csr_tensor(torch.from_numpy(rp), torch.from_numpy(ci.astype(np.int64)),
                                     torch.from_numpy(vv), size=(n, n), dtype=torch.float64, device="cuda")

        def mv(P, W):
            W.copy_(torch.sparse.mm(Qt, P))
        mf = L.ld_create_matfree(n, mv, col, lo, hi, 20, 1e-6)
        timed_evals(L, mf, 1)
        r = timed_evals(L, mf, 1)
        mi = r["info"]
        res["matfree_fp64"] = {"value": 1.0 / (r["ms"] / 1e3), "iters": mi["iters"],
                               "launches_per_iter": mi["gpu_launches"] / max(mi["iters"], 1),
                               "ms_per_iter": r["ms"] / max(mi["iters"], 1),
                               "logdet_rel_diff": abs(r["logdet"] - f["logdet"]) / abs(f["logdet"]) if f else None,
                               "callback": "torch.sparse.mm on a CSR tensor (cuSPARSE SpMM) + copy"}
        del mf
    return res


def run_mesh(args):
    """The general-mesh workload alone (--side vertices a side, 1024 by default), one line."""
    import torch
    import paper_1105_5256_gb300 as L
    torch.cuda.set_device(0)
    L.library(build_if_missing=True)
    peak, src = peak_hbm()
    side = args.side or 1024
    r = config_mesh(L, side, max(args.steps, 1), peak, src, matfree=args.fp64_sample > 0,
                    fp64=args.fp64_sample > 0, T=args.tile_width)
    line = {"metric": "log-det evals/sec (FEM SPDE alpha=2 on a %d^2-vertex mesh, CSR, d=2, N=20)" % side,
            "value": r.pop("value"), "unit": UNIT, "n_gpus": 1, "steps": r["evaluations"], "warmup": 1,
            "higher_is_better": True, "dtype": r.pop("dtype"), "data": "synthetic (seeded mesh)",
            "config": {"workload": r.pop("workload")}}
    line.update(r)
    print(json.dumps(line), flush=True)


def config_batch(L, steps, warmup, peak, src, fp64=True):
    """The batch workload: 256 independent 2D GMRFs of uneven size (sides 32..512, 5-point d=4 or
    13-point d=2, kappa^2 log-uniform) in one persistent launch per step; mixed precision,
    with (fp64) the same batch in the plain FP64 form and 256 sequential FP64 ld_logdet calls
    (one context per instance) beside it."""
    insts = synth.batch_instances(3, count=256)
    mats = [L.grid_matrix(i.kind, i.dims, i.kappa2) for i in insts]
    dists = [i.distance for i in insts]
    out = {}
    for name, prec in (("mixed", L.LD_MIXED), ("fp64", L.LD_FP64)):
        if name == "fp64" and not fp64:
            continue
        b = L.ld_batch_create(mats, dists, NSHIFT, TOL, L.options(precision=prec))
        for _ in range(warmup):
            L.ld_batch_logdet(b)
        ms = 0.0
        vti = 0
        for _ in range(steps):
            vals, _, info = L.ld_batch_logdet(b)
            ms += info["ms"]
            vti += info["vertex_tile_iters"]
        word = 4 if prec == L.LD_MIXED else 8
        # the active bytes: 4 state words a vertex and column of every pass each tile ran
        alg = 4 * word * info["tile_width"] * vti
        achieved = alg / (ms / 1e3) / 1e9
        out[name] = {"value": 256 * steps / (ms / 1e3), "ms_per_step": ms / steps,
                     "vals": vals, "tile_width": info["tile_width"],
                     "roofline": {"bound": "hbm", "kernel": "k_batch_solve + grid engine (large instances)",
                                  "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                  "traffic": None, "algorithmic_bytes_per_step": alg / steps,
                                  "peak_source": src,
                                  "note": "whole batch wall time, both engines, over the active bytes"}}
        del b
    res = {"workload": "256 grids, sides U{32..512}, 5-pt d=4 / 13-pt d=2, N=20, tol 1e-6",
           "value": out["mixed"]["value"], "unit": UNIT, "evaluations": 256 * steps,
           "ms_per_step": out["mixed"]["ms_per_step"], "dtype": "f32 vectors / f64 scalars",
           "points": int(sum(i.n for i in insts)), "tile_width": out["mixed"]["tile_width"],
           "roofline": out["mixed"]["roofline"]}
    if fp64:
        # 256 sequential FP64 evaluations, one context per instance (created beforehand)
        ctxs = [L.ld_create(m, d, NSHIFT, TOL, L.options(precision=L.LD_FP64)) for m, d in zip(mats, dists)]
        seq_ms, seq_vals = 0.0, []
        for c in ctxs:
            v, info = L.ld_logdet(c)
            seq_ms += info["ms"]
            seq_vals.append(v)
        del ctxs
        seq_vals = np.array(seq_vals)
        rel = float(np.max(np.abs(out["mixed"]["vals"] - out["fp64"]["vals"]) / np.abs(out["fp64"]["vals"])))
        rel_seq = float(np.max(np.abs(out["mixed"]["vals"] - seq_vals) / np.abs(seq_vals)))
        res["fp64_form"] = {"value": out["fp64"]["value"], "ms_per_step": out["fp64"]["ms_per_step"],
                            "mixed_vs_fp64_rel_diff_max": rel, "roofline": out["fp64"]["roofline"]}
        res["sequential_fp64"] = {"value": 256 / (seq_ms / 1e3), "ms": seq_ms,
                                  "note": "256 separate ld_logdet calls in FP64, one context per instance",
                                  "mixed_batch_vs_sequential_rel_diff_max": rel_seq}
    return res


def run_batch(args):
    """The batch workload alone, one JSON line (`--fp64-sample 0` skips the FP64 arms)."""
    import torch
    import paper_1105_5256_gb300 as L
    torch.cuda.set_device(0)
    L.library(build_if_missing=True)
    peak, src = peak_hbm()
    r = config_batch(L, args.steps, args.warmup, peak, src, fp64=args.fp64_sample > 0)
    line = {"metric": "log-det evals/sec (batch of 256 uneven 2D GMRFs, one persistent launch)",
            "value": r.pop("value"), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": r.pop("dtype"), "data": "synthetic (seeded batch)",
            "config": {"workload": r.pop("workload"), "points": r.pop("points"),
                       "tile_width": r.pop("tile_width")}}
    r.pop("unit")
    r.pop("evaluations")
    line.update(r)
    print(json.dumps(line), flush=True)


def run_small_configs(args):
    """The small CSR workload and the 2048^2 posterior, one JSON line each."""
    import torch
    import paper_1105_5256_gb300 as L
    torch.cuda.set_device(0)
    L.library(build_if_missing=True)
    peak, src = peak_hbm()
    for fn, metric in ((lambda: config_periodic64(L, max(args.steps, 10)),
                        "log-det evals/sec (64^2 periodic 5-point as CSR, d=4, N=20, FP64)"),
                       (lambda: config_posterior2048(L, max(args.steps, 2), peak, src),
                        "log-det+grad evals/sec (2048^2 Gauss-linear posterior, d=4, N=20)")):
        r = fn()
        line = {"metric": metric, "value": r.pop("value"), "unit": UNIT, "n_gpus": 1, "steps": r["evaluations"],
                "warmup": 1, "higher_is_better": True, "dtype": r.pop("dtype"), "data": "synthetic",
                "config": {"workload": r.pop("workload")}}
        line.update(r)
        print(json.dumps(line), flush=True)


def run_periodic64(args):
    """The 64^2 torus as CSR (FP64) alone, one JSON line."""
    import torch
    import paper_1105_5256_gb300 as L
    torch.cuda.set_device(0)
    L.library(build_if_missing=True)
    r = config_periodic64(L, max(args.steps, 1))
    line = {"metric": "log-det evals/sec (64^2 periodic 5-point as CSR, d=4, N=20, FP64)", "value": r.pop("value"),
            "unit": UNIT, "n_gpus": 1, "steps": r["evaluations"], "warmup": 2, "higher_is_better": True,
            "dtype": r.pop("dtype"), "data": "synthetic", "config": {"workload": r.pop("workload")}}
    line.update(r)
    print(json.dumps(line), flush=True)


def run_posterior(args):
    """The 2048^2 posterior alone (mixed with reliable updates, gradient), one
    JSON line; `--steps 1 --warmup 0 --fp64-sample 0` runs a single evaluation."""
    import torch
    import paper_1105_5256_gb300 as L
    torch.cuda.set_device(0)
    L.library(build_if_missing=True)
    peak, src = peak_hbm()
    r = config_posterior2048(L, max(args.steps, 1), peak, src, warmup=args.warmup, fp64=args.fp64_sample > 0)
    line = {"metric": "log-det+grad evals/sec (2048^2 Gauss-linear posterior, d=4, N=20)", "value": r.pop("value"),
            "unit": UNIT, "n_gpus": 1, "steps": r["evaluations"], "warmup": args.warmup, "higher_is_better": True,
            "dtype": r.pop("dtype"), "data": "synthetic", "config": {"workload": r.pop("workload")}}
    line.update(r)
    print(json.dumps(line), flush=True)


def run_field3d(args):
    """The 3D field (Dirichlet 256^3 by default, `--side` for smaller grids), one JSON line."""
    import torch
    import paper_1105_5256_gb300 as L
    torch.cuda.set_device(0)
    L.library(build_if_missing=True)
    peak, src = peak_hbm()
    clocks = Clocks()
    clocks.start()
    t0 = time.perf_counter()
    side = args.side or 256
    r = config_field3d(L, side, args.steps, peak, src, fp64=args.fp64_sample > 0, T=args.tile_width)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    line = {"metric": "log-det+grad evals/sec (Dirichlet %d^3, 7-point, kappa^2 field, d=6, N=32)" % side,
            "value": r.pop("value"), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": r.pop("dtype"),
            "data": "synthetic (seeded kappa^2 field)", "config": {"workload": r.pop("workload")},
            "clocks": clk, "wall_s": wall}
    line.update(r)
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
    split = args.split == "colours" and ws > 1
    prec = L.LD_MIXED if args.precision == "mixed" else L.LD_FP64
    # weak scaling: a seeded batch per rank; colour split: every rank the same batch
    draws = rank_draws(0 if split else rank, args.batch)
    if args.kappa2 > 0:
        draws = np.full(args.batch, args.kappa2)
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D13_SQ, DIMS, float(draws[0])), DIST, NSHIFT,
                      TOL, L.options(precision=prec, tile_width=args.tile_width))
    n = DIMS[0] * DIMS[1]
    ncol_all = L.ld_get_colouring(ctx)[1]
    cb, ce = colour_ranges(ncol_all, ws)[rank] if split else (0, ncol_all)

    def step():
        infos = []
        vals = []
        for k2 in draws:
            L.ld_set_params(ctx, float(k2))
            if split:
                v, info = L.ld_logdet_partial(ctx, cb, ce)
                v = combine_partials([v])[0]
            else:
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
    dev_ms = iter_ms = 0.0
    tile_iters = launches = passes = 0
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
            passes += i["iters"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    if ws > 1:   # max over ranks of device and wall time
        t = torch.tensor([dev_ms, wall], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dev_ms, wall = float(t[0]), float(t[1])
    evals = args.batch * args.steps * (1 if split else ws)
    value = evals / (dev_ms / 1e3)
    e2e = evals / wall
    info0 = all_infos[0]
    T = info0["tile_width"]
    ncols = ((info0["n_colours"] + T - 1) // T) * T
    word = 4 if args.precision == "mixed" else 8
    peak, src = peak_hbm()
    r = {"tile_iters": tile_iters, "passes": passes, "iter_ms": iter_ms, "info": all_infos[-1]}
    if args.precision == "fp64":
        # FP64 issue-bound: 25 flops per vertex-column per pass against the measured
        # 1.25 TFLOP/s non-tensor FP64 rate
        flops = FP64_FLOPS_PER_VC * n * T * tile_iters
        roof = {"bound": "alu", "kernel": "k_stream2d (stored-w pass, FP64)",
                "achieved": flops / (iter_ms / 1e3) / 1e9, "peak": FP64_PEAK_GFLOPS,
                "unit": "GFLOP/s", "traffic": None,
                "peak_source": "measured FP64 FMA-chain rate (equals the nominal 1.25 TFLOP/s)"}
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        lean = info0["pass_words"] == 4
        roof = roofline_entry("k_lean2d (lean fused CG pass, Matern square)" if lean else
                              "k_stream2d (stored-w fused CG pass)", n, T, word, r, False, 0, peak, src,
                              traffic=recorded_traffic("k_lean2d_matern1024_T2.md") if lean and T == 2 else None)
        roof["launch"] = ("one CG pass: the %d tile launches of an iteration, run concurrently on their "
                          "own streams" % (ncols // T))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if split else "weak", "vs_baseline": None,
        "dtype": "f32 vectors / f64 scalars" if args.precision == "mixed" else "f64",
        "data": "synthetic (seeded kappa^2 draws; no dataset)",
        "config": {"workload": "Matern alpha=2 (kappa^2 I - Lap)^2, 1024x1024 Dirichlet, 13-point",
                   "n": n, "colouring_distance": DIST, "n_colours": info0["n_colours"],
                   "n_shifts": NSHIFT, "tol": TOL, "batch_kappa2_draws": args.batch,
                   "precision": args.precision, "tile_width": T, "engine": info0["engine"],
                   "parallelism": ("colour split over %d ranks" % ws) if split else
                                  "dp%d (independent batches)" % ws,
                   "l2": "a CG pass streams %.2f GB of state > 129 MB L2 (no flush needed)"
                         % (info0["pass_words"] * n * ncols * word / 1e9)},
        "clocks": clk,
        "e2e": {"value": e2e, "unit": UNIT,
                "h2d_bytes_per_step": args.batch * (3 * 8 + 2 * NSHIFT * 16),
                "d2h_bytes_per_step": args.batch * (2 * 8 + 2 * 4 + 4 * ncols)},
        "gpu_launches": launches,
        "roofline": roof,
        "iters_mean": float(np.mean([i["iters"] for i in all_infos])),
        "logdet_first": vals[0],
    }
    if rank == 0 and ws == 1 and args.precision == "mixed" and args.fp64_sample > 0:
        out["fp64_form"] = fp64_form(L, draws[:args.fp64_sample], vals[:args.fp64_sample])
    if rank == 0 and ws == 1 and not args.no_other_configs:
        oc = {}
        for key, fn in (("periodic64_csr_fp64", lambda: config_periodic64(L, 10)),
                        ("posterior2048_mixed_grad", lambda: config_posterior2048(L, 3, peak, src)),
                        ("field3d256_mixed_grad", lambda: config_field3d(L, 256, 1, peak, src)),
                        ("mesh1024_csr_mixed", lambda: config_mesh(L, 1024, 2, peak, src)),
                        ("batch256_mixed", lambda: config_batch(L, 2, 1, peak, src, fp64=False))):
            try:
                oc[key] = fn()
            except Exception as e:      # a failing side configuration must not lose the headline
                oc[key] = {"error": str(e)[:300]}
        out["other_configs"] = oc
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


# ---------------------------------------------------------------- CPU baselines (the oracle)
def _o1_block_seconds(lines: int, k2: float) -> float:
    """Seconds of the oracle's banded Cholesky log det on the leading 1024 x lines block of
    the Matern precision (one core)."""
    from oracle import matrices as om
    from oracle import method as mt
    Qs = om.precision(om.KIND_2D13_SQ, (DIMS[0], lines), k2)
    t0 = time.perf_counter()
    mt.exact_logdet_band(Qs)
    return time.perf_counter() - t0


def _o4_colour_seconds(args) -> float:
    """Seconds of the oracle's CG-M method reference for one probing vector (one core)."""
    side, k2, colour_id = args
    from oracle import matrices as om
    from oracle import method as mt
    from oracle import probing
    Q = om.precision(om.KIND_2D13_SQ, (side, side), k2)
    col = probing.colour_greedy(Q, DIST)
    lo, hi = mt.spectral_bounds(om.KIND_2D13_SQ, (side, side), k2)
    t0 = time.perf_counter()
    mt.logdet_method(Q, col, lo, hi, NSHIFT, TOL, per_colour=True, colours=[colour_id])
    return time.perf_counter() - t0


def cpu_baseline(budget_s: float):
    """The oracle timed on the host cores, on bounded samples of the same workload.

    O1 (the traditional method of Sec. 2: plain natural-order banded Cholesky, log det =
    2 sum log L_jj) on a 1024 x k leading block (k doubled from 4 until the run takes a
    sixth of the budget), on one core, then one block per core at once (independent
    evaluations, as the batch of kappa^2 draws is); its cost is linear in the rows at fixed
    band, so the full-size time is projected by n / rows.  O4 (the method itself on the
    CPU: colouring, rational nodes and CG-M in numpy) runs every probing vector of a
    128 x 128 instance, the colours spread over the cores; it is projected to 1024^2 by the
    vertex count (the iteration count depends on kappa^2, not on the grid size, once the
    grid is larger than the correlation length)."""
    import multiprocessing as mpx
    k2 = float(synth.kappa2_draws(SEED, BATCH)[0])
    n = DIMS[0] * DIMS[1]
    cores = len(os.sched_getaffinity(0))
    lines = 4
    while True:
        dt = _o1_block_seconds(lines, k2)
        if dt > budget_s / 6 or lines >= DIMS[1]:
            break
        lines *= 2
    rows = DIMS[0] * lines
    single = 1.0 / (dt * n / rows)
    ctx = mpx.get_context("spawn")
    # one BLAS thread per worker process (the workers are the parallelism)
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({k: "1" for k in saved})
    with ctx.Pool(cores) as pool:
        t0 = time.perf_counter()
        per = pool.starmap(_o1_block_seconds, [(lines, k2)] * cores)
        wall_all = time.perf_counter() - t0
        all_rate = cores / (max(per) * n / rows)
        side = 128
        from oracle import matrices as om
        from oracle import probing
        C = int(probing.colour_greedy(om.precision(om.KIND_2D13_SQ, (side, side), k2), DIST).max()) + 1
        t0 = time.perf_counter()
        pool.map(_o4_colour_seconds, [(side, k2, c) for c in range(C)])
        o4_wall = time.perf_counter() - t0
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    o4_rate = 1.0 / o4_wall
    return {"value": all_rate, "unit": UNIT, "cores": cores, "kind": "oracle", "projected": True,
            "sample": "O1 banded Cholesky log det of the same model on a %dx%d block (%d rows, band %d), "
                      "one block per core at once, %.2f s each (slowest), projected by n/rows = %.0f"
                      % (DIMS[0], lines, rows, 2 * DIMS[0], max(per), n / rows),
            "single_core": {"value": single, "unit": UNIT, "cores": 1, "projected": True,
                            "sample_seconds": dt},
            "cores_all": {"value": all_rate, "unit": UNIT, "cores": cores, "projected": True,
                          "sample_seconds_max": max(per), "wall_s": wall_all},
            "o4": {"value_128": o4_rate, "unit": UNIT, "cores": cores, "sample_seconds": o4_wall,
                   "value": o4_rate / (n / side ** 2), "projected": True,
                   "sample": "CG-M method reference (colouring d=2, N=20, tol 1e-6) on the 128x128 "
                             "Matern instance, %d colours over %d cores, projected by n ratio %d"
                             % (C, cores, n // side ** 2)}}


def run_reference(args):
    """The reference arm: the oracle (banded Cholesky, the traditional route of Sec. 2) as it
    stands, on the host cores, on bounded samples of the same workload; one step = one
    sample run on every core at once, reported as projected full-size evaluations/s."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mpx
    k2 = float(synth.kappa2_draws(SEED, BATCH)[0])
    n = DIMS[0] * DIMS[1]
    cores = len(os.sched_getaffinity(0))
    lines = 4
    while True:
        dt = _o1_block_seconds(lines, k2)
        if dt > args.cpu_seconds / 6 or lines >= DIMS[1]:
            break
        lines *= 2
    rows = DIMS[0] * lines
    ctx = mpx.get_context("spawn")
    step_s, rates = [], []
    os.environ.update({k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")})
    with ctx.Pool(cores) as pool:
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            per = pool.starmap(_o1_block_seconds, [(lines, k2)] * cores)
            if k >= args.warmup:
                step_s.append(time.perf_counter() - t0)
                rates.append(cores / (max(per) * n / rows))
    value = statistics.mean(rates)
    sample = ("O1 banded Cholesky log det of the same model on a %dx%d block (%d rows, band %d), one "
              "block per core on %d cores, projected by n/rows = %.0f" % (DIMS[0], lines, rows, 2 * DIMS[0],
                                                                         cores, n / rows))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_s) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "projected": True,
           "config": {"workload": "Matern alpha=2 (kappa^2 I - Lap)^2, 1024x1024 Dirichlet, 13-point"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample, "projected": True},
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
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the other configurations (profiling runs)")
    ap.add_argument("--batch", type=int, default=BATCH, help="kappa^2 values per step")
    ap.add_argument("--tile-width", type=int, default=0, help="probing vectors per tile (0 = auto)")
    ap.add_argument("--split", default="batches", choices=["batches", "colours"],
                    help="several GPUs: independent batches per rank, or every evaluation's colours split")
    ap.add_argument("--workload", default="matern1024",
                    choices=["matern1024", "batch256", "field3d256", "small", "posterior2048", "mesh1024",
                             "periodic64"])
    ap.add_argument("--side", type=int, default=0,
                    help="grid side (field3d256 workload, default 256) or mesh vertices a side (mesh1024, "
                         "default 1024)")
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
    elif args.workload == "posterior2048":
        run_posterior(args)
    elif args.workload == "mesh1024":
        run_mesh(args)
    elif args.workload == "periodic64":
        run_periodic64(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
