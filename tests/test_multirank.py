"""Multi-process (world size 2, gloo, CPU) checks of the sharding logic.

The path shards by independent problems (each rank evaluates its own seeded
kappa^2 batch, no data-path collective) or, for one evaluation, by colour ranges
whose partial sums add up (the paper's one-probing-vector-per-node scheme,
Sec. 2.1).  These tests run the host-side logic in two gloo processes.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    draws = bench.rank_draws(rank, 16)
    got = [None] * world
    dist.all_gather_object(got, [float(x) for x in draws])
    # colour ranges of one evaluation split across ranks
    ranges = bench.colour_ranges(18, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, ranges[rank])
    # max-over-ranks timing
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((got, gathered, float(t[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got, gathered, tmax = q.get(timeout=120)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got[0] != got[1]                       # independent seeded batches
    assert np.allclose(got[0], bench.rank_draws(0, 16))
    cover = sorted(c for a, b in gathered for c in range(a, b))
    assert cover == list(range(18))               # colour ranges partition [0, C)
    assert tmax == 2.0                            # the slowest rank sets the time


def _partial_worker(rank, world, port, q):
    """One rank of a colour-split evaluation: the per-colour terms (and seed projections,
    the kappa^2 gradient terms) of its colour range, summed locally and combined by the
    bench's all-reduce.  The terms come from a CPU stand-in (the oracle's circulant
    probed values of a periodic grid), so the combine path runs without a GPU."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import closed_forms as cf
    from oracle import hht
    from oracle import matrices as om
    from oracle import method as mt
    from oracle import probing
    dims, k2 = (24, 20), 0.3
    col = probing.colour_greedy(om.precision(om.KIND_2D5, dims, k2, periodic=True), 4)
    lo, hi = mt.spectral_bounds(om.KIND_2D5, dims, k2, periodic=True)
    s, a = hht.log_nodes(lo, hi, 20)
    terms = cf.probed_value(om.KIND_2D5, dims, k2, True, col, lambda lam: hht.f_N(lam, s, a), per_colour=True)
    seeds = cf.probed_value(om.KIND_2D5, dims, k2, True, col, lambda lam: 1.0 / lam, per_colour=True)
    cb, ce = bench.colour_ranges(len(terms), world)[rank]
    total = bench.combine_partials([float(np.sum(terms[cb:ce])), float(np.sum(seeds[cb:ce]))])
    if rank == 0:
        q.put((total, float(np.sum(terms)), float(np.sum(seeds)), len(terms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_colour_split_combines_partials():
    """Sec. 2.1's one-probing-vector-per-node scheme: the partial log det and gradient of
    two colour ranges, combined by one all-reduce, equal the single-rank sums to 1e-14."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_partial_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    (ld, g), ld_ref, g_ref, C = q.get(timeout=120)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert C > 2
    assert abs(ld - ld_ref) <= 1e-14 * abs(ld_ref)
    assert abs(g - g_ref) <= 1e-14 * abs(g_ref)


def test_colour_ranges_cover_and_balance():
    for C in (1, 5, 18, 107):
        for world in (1, 2, 3, 8):
            rs = bench.colour_ranges(C, world)
            assert len(rs) == world
            assert rs[0][0] == 0 and rs[-1][1] == C
            assert all(a <= b for a, b in rs)
            assert all(rs[k][1] == rs[k + 1][0] for k in range(world - 1))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle on the host, no GPU) prints one JSON line with the
    contract's keys; the e2e record of a host program moves no bytes."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                          "--cpu-seconds", "0.4"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]
