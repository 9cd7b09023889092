"""Host-side checks of liblogdet (no GPU): the library loads, exports every entry
point the header declares, and its host steps match the oracle.

  * colouring (Sec. 2.1, greedy distance-d, natural order) -- bit-exact;
  * quadrature nodes and weights (Eq. "eq_rat_app")        -- to 1e-12;
  * spectral interval                                      -- to 1e-14.
"""
import os
import re

import numpy as np
import scipy.sparse as sp
import pytest

import paper_1105_5256_gb300 as L
import synth
from oracle import hht
from oracle import matrices as om
from oracle import method as mt
from oracle import probing

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "logdet.h")).read()
    return sorted(set(re.findall(r"^\s*(?:ld_status|int|void|const char \*)\s*\*?\s*(ld_\w+)\s*\(",
                                 src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    syms = header_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), s
    assert lib.ld_abi_version() == 6


@pytest.mark.parametrize("kind,dims,per,d", [
    (om.KIND_2D5, (64, 64), True, 4),
    (om.KIND_2D5, (64, 64), True, 2),
    (om.KIND_2D5, (57, 31), False, 4),
    (om.KIND_2D5, (1, 40), False, 3),
    (om.KIND_2D5, (3, 5), True, 2),
    (om.KIND_2D13_SQ, (40, 37), False, 2),
    (om.KIND_2D13_SQ, (12, 12), True, 1),
    (om.KIND_3D7, (9, 8, 7), False, 3),
    (om.KIND_3D7, (6, 6, 6), True, 2),
])
def test_grid_colouring_bit_exact(lib, kind, dims, per, d):
    Q = om.precision(kind, dims, 0.5, periodic=per)
    ref = probing.colour_greedy(Q, d)
    col, nc = L.ld_colour_grid(kind, dims, per, d)
    assert np.array_equal(col, ref)
    assert nc == int(ref.max()) + 1


def test_grid_colouring_random_shapes_bit_exact(lib):
    """Seeded sweep over kinds, torus or Dirichlet, thin and tiny grids and distances 0-6:
    the lattice colouring (fast interior path plus the bounds-checked edge path) equals the
    oracle's breadth-first greedy colouring everywhere."""
    rng = np.random.default_rng(7)
    for trial in range(150):
        kind = [om.KIND_2D5, om.KIND_2D13_SQ, om.KIND_3D7][trial % 3]
        per = bool(rng.integers(0, 2))
        nd = 3 if kind == om.KIND_3D7 else 2
        dims = tuple(int(v) for v in rng.integers(1, 13 if nd == 3 else 40, size=nd))
        d = int(rng.integers(0, 7))
        ref = probing.colour_greedy(om.precision(kind, dims, 0.5, periodic=per), d)
        col, nc = L.ld_colour_grid(kind, dims, per, d)
        assert np.array_equal(col, ref), (kind, dims, per, d)
        assert nc == int(ref.max()) + 1


def test_csr_colouring_bit_exact(lib):
    n = 700
    rows, cols, w = synth.random_sparse_spd_pattern(11, n)
    rp, ci, vv = synth.csr_from_edges(n, rows, cols, w, 0.5)
    import scipy.sparse as sp
    Q = sp.csr_matrix((vv, ci, rp), shape=(n, n))
    for d in (1, 2, 3):
        ref = probing.colour_greedy(Q, d)
        col, nc = L.ld_colour_csr(rp, ci, d)
        assert np.array_equal(col, ref)


@pytest.mark.parametrize("m,M,N", [(0.5, 8.5, 20), (1e-4, 64.2, 20), (0.01, 12.0, 32),
                                   (1.0, 1.01, 4), (3.0, 3e6, 40)])
def test_nodes_match_oracle(lib, m, M, N):
    s, a, cert = L.ld_hht_nodes(m, M, N)
    so, ao = hht.log_nodes(m, M, N)
    assert np.abs(s - so).max() <= 1e-12 * np.abs(so).max()
    assert np.abs(a - ao).max() <= 1e-12 * np.abs(ao).max()
    co = hht.certificate(m, M, so, ao, samples=2001)
    assert abs(cert - co) <= 1e-12 + 1e-6 * co


@pytest.mark.parametrize("m,M,N", [(0.5, 8.5, 20), (1e-4, 64.2, 24), (3.0, 3e6, 40)])
def test_invsqrt_nodes_match_oracle(lib, m, M, N):
    s, b = L.ld_hht_invsqrt_nodes(m, M, N)
    so, bo = hht.invsqrt_nodes(m, M, N)
    assert np.abs(s - so).max() <= 1e-12 * np.abs(so).max()
    assert np.abs(b - bo).max() <= 1e-12 * np.abs(bo).max()


def test_node_errors(lib):
    with pytest.raises(L.LogDetError):
        L.ld_hht_nodes(-1.0, 2.0, 8)
    with pytest.raises(L.LogDetError):
        L.ld_hht_nodes(1.0, 2.0, 0)


@pytest.mark.parametrize("kind,dims,per,k2,tau,masked,scale", [
    (om.KIND_2D5, (64, 64), True, 0.5, 0.0, False, 1.0),
    (om.KIND_2D5, (100, 37), False, 0.1, 4.0, True, 1.0),
    (om.KIND_2D13_SQ, (1024, 1024), False, 0.01, 0.0, False, 2.0),
    (om.KIND_3D7, (16, 12, 9), False, 0.3, 0.0, False, 0.7),
])
def test_bounds_match_oracle(lib, kind, dims, per, k2, tau, masked, scale):
    n = int(np.prod(dims))
    mask = synth.obs_mask(4, n, 0.1) if masked else None
    lo, hi = L.ld_grid_bounds(L.grid_matrix(kind, dims, k2, periodic=per, tau=tau, obs_mask=mask,
                                            scale=scale))
    lo_o, hi_o = mt.spectral_bounds(kind, dims, k2, periodic=per, tau=tau, mask=mask, scale=scale)
    assert abs(lo - lo_o) <= 1e-14 * lo_o and abs(hi - hi_o) <= 1e-14 * hi_o


def test_field_bounds_match_oracle(lib):
    dims = (10, 9, 8)
    f = synth.kappa2_field(5, dims)
    lo, hi = L.ld_grid_bounds(L.grid_matrix(om.KIND_3D7, dims, 1.0, kappa2_field=f))
    lo_o, hi_o = mt.spectral_bounds(om.KIND_3D7, dims, f)
    assert abs(lo - lo_o) <= 1e-14 * lo_o and abs(hi - hi_o) <= 1e-14 * hi_o


def test_invalid_matrix_rejected_on_host(lib):
    with pytest.raises(L.LogDetError) as e:
        L.ld_grid_bounds(L.grid_matrix(om.KIND_2D5, (0, 4), 0.5))
    assert e.value.status == L.LD_EINVAL
    with pytest.raises(L.LogDetError) as e:
        L.ld_grid_bounds(L.grid_matrix(om.KIND_2D13_SQ, (8, 8), 0.5, kappa2_field=np.ones(64)))
    assert e.value.status == L.LD_EUNSUPPORTED


@pytest.mark.parametrize("kw", [{"reliable_delta": 1.5}, {"reliable_delta": -0.1}, {"engine": 3},
                                {"chunk_iters": -1}, {"precision": 7}])
def test_invalid_options_rejected_before_any_device_work(lib, kw):
    """Option checks run before the context touches the device (no GPU needed)."""
    with pytest.raises(L.LogDetError) as e:
        L.ld_create(L.grid_matrix(om.KIND_2D5, (8, 8), 0.5), 2, 8, 1e-8, L.options(**kw))
    assert e.value.status == L.LD_EINVAL


@pytest.mark.parametrize("seed,n,shift", [(21, 600, 0.2), (3, 2000, 0.01), (8, 50, 1.0)])
def test_csr_bounds_enclose_the_spectrum(lib, seed, n, shift):
    """Host bound estimate for CSR: Gershgorin above lambda_max; half the converged smallest
    Lanczos Ritz value below lambda_min (and within a factor 4 of it), against eigvalsh."""
    rows, cols, w = synth.random_sparse_spd_pattern(seed, n)
    rp, ci, vv = synth.csr_from_edges(n, rows, cols, w, shift)
    ev = np.linalg.eigvalsh(sp.csr_matrix((vv, ci, rp), shape=(n, n)).toarray())
    lo, hi = L.ld_csr_bounds(rp, ci, vv, 1.5)
    assert hi >= 1.5 * ev.max() * (1 - 1e-12)
    assert 1.5 * ev.min() / 4 <= lo <= 1.5 * ev.min()


@pytest.mark.parametrize("case", ["fem2_k0.5", "fem2_k0.01", "fem2_61", "matern_1e-4"])
def test_csr_bounds_converge_on_ill_conditioned_matrices(lib, case):
    """Condition numbers 1e6 to 1e12 need thousands of Lanczos steps (more than n for the
    smaller ones): the lower bound must still be half the smallest eigenvalue, i.e. the
    Ritz value converged instead of stopping at a fixed step count."""
    if case.startswith("fem2"):
        nx, k2 = (61, 10.0) if case == "fem2_61" else (31, float(case.split("_k")[1]))
        p, t = synth.perturbed_triangulation(11, nx, nx - 4 if nx == 31 else nx)
        Q = om.fem_spde_precision(p, t, k2, 2)
    else:
        Q = om.precision(om.KIND_2D13_SQ, (60, 60), 1e-4)
    rp, ci, vv = om.csr_arrays(Q)
    ev = np.linalg.eigvalsh(Q.toarray())
    lo, hi = L.ld_csr_bounds(rp, ci, vv)
    assert hi >= ev.max() * (1 - 1e-12)
    assert 0.49 * ev.min() <= lo <= 0.5 * ev.min() * (1 + 1e-3)


def test_csr_bounds_unconverged_is_an_error_not_a_guess(lib):
    """A 1D chain with kappa^2 = 1e-8 (condition number about 4e8, 2e4 Lanczos steps) and
    200k vertices: the host step budget runs out first, so the bound fails with LD_ENOTCONV
    and ld_create asks for user bounds instead of using an unconverged estimate."""
    n = 200_000
    rows = np.arange(1, n, dtype=np.int64)
    rp, ci, vv = synth.csr_from_edges(n, rows, rows - 1, np.ones(n - 1), 1e-8)
    with pytest.raises(L.LogDetError) as e:
        L.ld_csr_bounds(rp, ci, vv)
    assert e.value.status == L.LD_ENOTCONV
    with pytest.raises(L.LogDetError) as e:
        L.ld_create(L.csr_matrix(rp, ci, vv), 1, 8, 1e-6)
    assert e.value.status == L.LD_ENOTCONV and "lambda_min" in L.ld_last_error()


def test_csr_bounds_reject_indefinite(lib):
    rp = np.array([0, 1, 2], dtype=np.int64)
    ci = np.array([0, 1], dtype=np.int32)
    with pytest.raises(L.LogDetError) as e:
        L.ld_csr_bounds(rp, ci, np.array([-1.0, -2.0]))
    assert e.value.status == L.LD_ENOTSPD


def test_matfree_create_checks_arguments_before_any_device_call(lib):
    """ld_create_matfree validates on the host (these run without a GPU)."""
    n = 50
    col = np.arange(n) % 3

    def mv(P, W):
        W.copy_(P)

    bad = [
        (dict(matvec=None), L.LD_EINVAL),
        (dict(colouring=-col - 1), L.LD_EINVAL),
        (dict(colouring=col + n), L.LD_EINVAL),
        (dict(lambda_min=0.0), L.LD_EINVAL),
        (dict(lambda_max=0.5), L.LD_EINVAL),
        (dict(lambda_max=np.inf), L.LD_EINVAL),
        (dict(n_shifts=0), L.LD_EINVAL),
        (dict(tol=0.0), L.LD_EINVAL),
        (dict(opts=L.options(precision=L.LD_MIXED)), L.LD_EUNSUPPORTED),
        (dict(opts=L.options(max_iter=-1)), L.LD_EINVAL),
    ]
    for kw, status in bad:
        args = dict(n=n, matvec=mv, colouring=col, lambda_min=1.0, lambda_max=2.0, n_shifts=8,
                    tol=1e-8, opts=None)
        args.update(kw)
        with pytest.raises(L.LogDetError) as e:
            L.ld_create_matfree(**args)
        assert e.value.status == status, kw


def test_matfree_derivative_setter_rejects_a_null_context(lib):
    """ld_matfree_set_derivative checks its context on the host."""
    fn = L.DMATVEC_FN(lambda *a: 0)
    assert lib.ld_matfree_set_derivative(None, fn, None, 1) == L.LD_EINVAL


def test_batch_create_checks_every_instance_on_the_host(lib):
    """ld_batch_create rejects bad shared arguments and bad instances before any device work."""
    good = [L.grid_matrix(om.KIND_2D5, (16, 16), 0.5), L.grid_matrix(om.KIND_2D13_SQ, (12, 9), 0.2)]
    rows, cols, w = synth.random_sparse_spd_pattern(1, 30)
    csr = L.csr_matrix(*synth.csr_from_edges(30, rows, cols, w, 0.5))
    cases = [
        (dict(tol=0.0), L.LD_EINVAL),
        (dict(n_shifts=0), L.LD_EINVAL),
        (dict(opts=L.options(precision=5)), L.LD_EINVAL),
        (dict(opts=L.options(max_iter=-2)), L.LD_EINVAL),
        (dict(distances=[2, -1]), L.LD_EINVAL),
        (dict(matrices=[good[0], csr]), L.LD_EUNSUPPORTED),
        (dict(matrices=[good[0], L.grid_matrix(om.KIND_2D5, (0, 5), 0.5)]), L.LD_EINVAL),
    ]
    for kw, status in cases:
        args = dict(matrices=good, distances=[2, 2], n_shifts=8, tol=1e-6, opts=None)
        args.update(kw)
        with pytest.raises(L.LogDetError) as e:
            L.ld_batch_create(**args)
        assert e.value.status == status, kw


def test_static_entry_point_rejects_before_any_device_work():
    """ld_logdet_static checks every size against its static scratch before it reads the
    colouring or touches a device: oversized grids (including vertex counts that would
    overflow) and bad arguments fail with LD_EINVAL on a machine with no GPU."""
    lib = L.library()
    m = L.grid_matrix(L.LD_STENCIL_2D5, (512, 512), 0.5)
    colour = np.zeros(512 * 512, dtype=np.int32)
    colour[-1] = -7                                  # never read: the size check comes first
    with pytest.raises(L.LogDetError) as e:
        L.ld_logdet_static(m, colour, 18, 20, 1e-8)
    assert e.value.status == L.LD_EINVAL and "LD_STATIC_SCRATCH_BYTES" in str(e.value)
    huge = L.grid_matrix(L.LD_STENCIL_3D7, (1 << 30, 1 << 30, 1 << 30), 0.5)
    with pytest.raises(L.LogDetError) as e:
        L.ld_logdet_static(huge, np.zeros(1, dtype=np.int32), 1, 20, 1e-8)
    assert e.value.status == L.LD_EINVAL and "LD_STATIC_SCRATCH_BYTES" in str(e.value)
    small = L.grid_matrix(L.LD_STENCIL_2D5, (8, 8), 0.5)
    for args in ((np.zeros(64, np.int32), 0, 20, 1e-8), (np.zeros(64, np.int32), 1, 0, 1e-8),
                 (np.zeros(64, np.int32), 1, 20, 0.0)):
        with pytest.raises(L.LogDetError) as e:
            L.ld_logdet_static(small, *args)
        assert e.value.status == L.LD_EINVAL
    assert lib is not None


def test_automatic_shift_count_meets_its_certificate_target():
    """n_shifts = 0 (Sec. 2.1's quadrature error rate): the library's N is the smallest whose
    certificate is at most 1e-10 |log M - log m|.  Against the oracle's nodes and its own
    certificate: N meets the target and N - 1 misses it (up to the two certificates'
    different sampling, a factor 2 at the boundary)."""
    from oracle import hht
    for kind, dims, k2 in ((L.LD_STENCIL_2D13_SQ, (64, 48), 0.01), (L.LD_STENCIL_2D5, (40, 30), 0.5),
                           (L.LD_STENCIL_3D7, (9, 8, 7), 0.2), (L.LD_STENCIL_2D13_SQ, (1024, 1024), 0.01)):
        lo, hi = L.ld_grid_bounds(L.grid_matrix(kind, dims, k2))
        target = 1e-10 * abs(np.log(hi) - np.log(lo))
        N = L.ld_auto_shifts(lo, hi)
        assert 4 < N < 256
        s, a = hht.log_nodes(lo, hi, N)
        assert hht.certificate(lo, hi, s, a) <= 2 * target
        s, a = hht.log_nodes(lo, hi, N - 1)
        assert hht.certificate(lo, hi, s, a) > 0.5 * target
    with pytest.raises(L.LogDetError):
        L.ld_auto_shifts(2.0, 1.0)


def test_package_import_requests_hardware_queues_for_its_streams():
    """Importing the package asks the CUDA runtime for 32 hardware queues (tile groups and a
    batch's concurrent instances run on streams of their own; with the default 8, streams
    beyond the eighth wait on one another), unless the caller set a value."""
    import subprocess
    import sys
    code = ("import os; os.environ.pop('CUDA_DEVICE_MAX_CONNECTIONS', None); "
            "import paper_1105_5256_gb300; print(os.environ['CUDA_DEVICE_MAX_CONNECTIONS'])")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-500:]
    assert out.stdout.strip() == "32"
    code2 = "import paper_1105_5256_gb300, os; print(os.environ['CUDA_DEVICE_MAX_CONNECTIONS'])"
    env = dict(os.environ, CUDA_DEVICE_MAX_CONNECTIONS="12")
    out2 = subprocess.run([sys.executable, "-c", code2], cwd=ROOT, capture_output=True, text=True, timeout=300,
                          env=env)
    assert out2.returncode == 0 and out2.stdout.strip() == "12"
