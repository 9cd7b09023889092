"""The allocation-free entry point ld_logdet_static agrees with ld_logdet.

ld_logdet_static serves callers that cannot allocate device memory (a
framework allocator or arena that owns all device memory, or a callback where
an allocation would synchronise the device): its work buffers live in the
library's static device array.  Here it is called twice in a row through the C
ABI on the same small model and compared with the allocating entry point, run
with the same engine (one CTA per probing vector, FP64, tile width 1), within
the FP64 parity tolerance the other GPU tests use; the device's free memory is
the same before and after the second call (the first call may load the
library's kernels).  This file is collected last so that a failure here never
hides another test's result.
"""
import numpy as np
import pytest

import paper_1105_5256_gb300 as L

pytestmark = pytest.mark.gpu

DIMS, KAPPA2, DIST, NSHIFT, TOL = (64, 64), 0.5, 4, 20, 1e-10


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


def test_static_matches_allocating_entry_point_twice():
    m = L.grid_matrix(L.LD_STENCIL_2D5, DIMS, KAPPA2, periodic=True)
    colour, nc = L.ld_colour_grid(L.LD_STENCIL_2D5, DIMS, True, DIST)
    ctx = L.ld_create(m, DIST, NSHIFT, TOL, L.options(engine=2, tile_width=1))
    ref, info = L.ld_logdet(ctx)
    terms, _ = L.ld_column_terms(ctx)
    bound = 50 * TOL * np.abs(terms).sum()
    import torch
    torch.cuda.synchronize()
    torch.cuda.mem_get_info()
    first = L.ld_logdet_static(m, colour, nc, NSHIFT, TOL)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    second = L.ld_logdet_static(m, colour, nc, NSHIFT, TOL)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, (free_before, free_after)   # nothing allocated
    assert abs(first - ref) <= bound
    assert abs(second - ref) <= bound
    assert first == second


def test_static_rejects_oversized_problem():
    m = L.grid_matrix(L.LD_STENCIL_2D5, (512, 512), KAPPA2)
    colour, nc = L.ld_colour_grid(L.LD_STENCIL_2D5, (512, 512), False, DIST)
    with pytest.raises(L.LogDetError) as e:
        L.ld_logdet_static(m, colour, nc, NSHIFT, TOL)
    assert e.value.status == L.LD_EINVAL
    assert "LD_STATIC_SCRATCH_BYTES" in str(e.value)
    # a colouring with an out-of-range entry is not even read when the grid is too large
    bad = colour.copy()
    bad[-1] = -5
    with pytest.raises(L.LogDetError) as e:
        L.ld_logdet_static(m, bad, nc, NSHIFT, TOL)
    assert "LD_STATIC_SCRATCH_BYTES" in str(e.value)
