"""General-mesh input on the host (no GPU): P1 finite-element SPDE precisions.

The oracle's assembly (one triangle at a time, hat gradients from inverting the
vertex matrix) is pinned to facts of the finite-element spaces themselves:
  * vertex quadrature is exact for linear functions: sum c = |domain|, c.x = integral x;
  * constants lie in the kernel of G: G 1 = 0;
  * linear functions are reproduced exactly: u^T G v = |domain| grad(u) . grad(v);
  * on the unperturbed square lattice (right isosceles triangles, either diagonal) the
    stiffness is the Neumann 5-point Laplacian, T (x) D + D (x) T, with T the 1D
    Neumann second difference and D = diag(1/2, 1, ..., 1, 1/2);
  * first-order matrix is SPD, the second-order one is K C~^{-1} K.
The library's native assembly (`ld_spde_fem_csr`, edge-vector formula) must equal the
oracle's, pattern included; the library's colouring and spectral interval run on the mesh
graph.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_1105_5256_gb300 as L
import synth
from oracle import matrices as om
from oracle import probing
from paper_1105_5256_gb300 import mesh


@pytest.fixture(scope="module")
def lib():
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


MESHES = [(3, 31, 27), (11, 17, 40)]


@pytest.mark.parametrize("seed,nx,ny", MESHES)
def test_triangulation_is_valid(seed, nx, ny):
    p, t = synth.perturbed_triangulation(seed, nx, ny)
    e1, e2 = p[t[:, 1]] - p[t[:, 0]], p[t[:, 2]] - p[t[:, 0]]
    area = 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    assert area.min() > 0 and abs(area.sum() - 1.0) < 1e-12
    assert p.min() == 0.0 and p.max() == 1.0
    # conforming: every interior edge is shared by exactly two triangles
    edges = np.sort(np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]]), axis=1)
    _, counts = np.unique(edges, axis=0, return_counts=True)
    assert set(counts.tolist()) <= {1, 2}
    assert (counts == 1).sum() == 2 * (nx - 1) + 2 * (ny - 1)


@pytest.mark.parametrize("seed,nx,ny", MESHES)
def test_oracle_fem_reproduces_linear_functions(seed, nx, ny):
    p, t = synth.perturbed_triangulation(seed, nx, ny)
    c, G = om.fem_p1(p, t)
    x, y = p[:, 0], p[:, 1]
    assert abs(c.sum() - 1.0) < 1e-13
    assert abs(c @ x - 0.5) < 1e-13 and abs(c @ y - 0.5) < 1e-13
    assert abs(G @ np.ones(len(c))).max() < 1e-12
    assert abs(G - G.T).max() < 1e-14
    rng = np.random.default_rng(0)
    for _ in range(3):
        a, b = rng.standard_normal(2), rng.standard_normal(2)
        u, v = p @ a, p @ b
        assert abs(u @ (G @ v) - a @ b) < 1e-11 * (1 + abs(a @ b))


@pytest.mark.parametrize("m", [6, 13])
def test_oracle_fem_regular_lattice_is_neumann_5_point(m):
    p, t = synth.perturbed_triangulation(5, m, m, jitter=0.0)
    c, G = om.fem_p1(p, t)
    T = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1]).tolil()
    T[0, 0] = T[m - 1, m - 1] = 1.0
    d = np.ones(m)
    d[0] = d[-1] = 0.5
    D = sp.diags(d)
    ref = sp.kron(T, D) + sp.kron(D, T)
    assert abs(G - ref).max() < 1e-12
    # lumped mass: a sixth of a cell per incident right triangle (the diagonals vary)
    h = 1.0 / (m - 1)
    inc = np.bincount(t.ravel(), minlength=m * m)
    assert np.allclose(c, inc * h * h / 6.0, rtol=1e-14, atol=0)


def test_oracle_spde_precisions():
    p, t = synth.perturbed_triangulation(3, 15, 12)
    c, G = om.fem_p1(p, t)
    Q1 = om.fem_spde_precision(p, t, 5.0, 1, 2.0)
    Q2 = om.fem_spde_precision(p, t, 5.0, 2, 2.0)
    K = (5.0 * sp.diags(c) + G).toarray()
    assert abs(Q1.toarray() - 2.0 * K).max() < 1e-13 * abs(K).max()
    assert abs(Q2.toarray() - 2.0 * K @ np.diag(1 / c) @ K).max() < 1e-12 * abs(Q2).max()
    for Q in (Q1, Q2):
        assert np.linalg.eigvalsh(Q.toarray()).min() > 0


@pytest.mark.parametrize("seed,nx,ny", MESHES)
@pytest.mark.parametrize("alpha", [1, 2])
def test_library_assembly_matches_oracle(seed, nx, ny, alpha):
    p, t = synth.perturbed_triangulation(seed, nx, ny)
    Qo = om.fem_spde_precision(p, t, 7.5, alpha, 0.5)
    rp, ci, vv = mesh.spde_csr(p, t, 7.5, alpha, 0.5)
    Qp = sp.csr_matrix((vv, ci, rp), shape=Qo.shape)
    assert abs(Qo - Qp).max() <= 1e-13 * abs(Qo).max()
    # either orientation of the triangles gives the same matrix
    rp2, ci2, vv2 = mesh.spde_csr(p, t[:, ::-1], 7.5, alpha, 0.5)
    assert abs(sp.csr_matrix((vv2, ci2, rp2), shape=Qo.shape) - Qp).max() <= 1e-13 * abs(Qo).max()


def test_library_assembly_rejects_bad_input(lib):
    p, t = synth.perturbed_triangulation(3, 5, 5)
    with pytest.raises(ValueError):
        mesh.spde_csr(p, t, 1.0, alpha=3)
    with pytest.raises(ValueError):
        mesh.spde_csr(p, t, 0.0)
    with pytest.raises(ValueError):
        mesh.spde_csr(p, t[:, :2], 1.0)
    bad = t.copy()
    bad[0] = [0, 1, 2]                       # three collinear vertices on the lower edge
    orphan = np.concatenate([p, [[0.5, 0.5]]])   # a vertex in no triangle
    for args in [(p, t + 100), (p, -t), (p, bad), (orphan, t)]:
        with pytest.raises(L.LogDetError) as e:
            mesh.spde_csr(*args, 1.0)
        assert e.value.status == L.LD_EINVAL
    # the C entry point checks its own arguments too (alpha, parameters, sizes)
    nnz = np.zeros(1, dtype=np.int64)
    P = np.ascontiguousarray(p)
    T = np.ascontiguousarray(t, dtype=np.int64)
    for a, k2, tau, n in [(3, 1.0, 1.0, len(p)), (1, -1.0, 1.0, len(p)), (1, 1.0, 0.0, len(p)),
                          (2, 1.0, 1.0, 2)]:
        st = lib.ld_spde_fem_csr(n, P.ctypes.data, len(T), T.ctypes.data, k2, a, tau, 0, None, None,
                                 None, nnz.ctypes.data_as(L.C.POINTER(L.C.c_int64)))
        assert st == L.LD_EINVAL


@pytest.mark.parametrize("seed,nx,ny", MESHES)
def test_library_assembly_query_then_fill(lib, seed, nx, ny):
    """Two-call protocol: a capacity below nnz writes only nnz; the filled CSR has sorted
    rows and the oracle's pattern exactly."""
    p, t = synth.perturbed_triangulation(seed, nx, ny)
    Q = om.fem_spde_precision(p, t, 2.0, 2)
    P = np.ascontiguousarray(p)
    T = np.ascontiguousarray(t, dtype=np.int64)
    nnz = np.zeros(1, dtype=np.int64)
    rp = np.full(len(p) + 1, -7, dtype=np.int64)
    ci = np.zeros(Q.nnz - 1, dtype=np.int32)
    vv = np.zeros(Q.nnz - 1)
    nptr = nnz.ctypes.data_as(L.C.POINTER(L.C.c_int64))
    assert lib.ld_spde_fem_csr(len(p), P.ctypes.data, len(T), T.ctypes.data, 2.0, 2, 1.0, Q.nnz - 1,
                               rp.ctypes.data, ci.ctypes.data, vv.ctypes.data, nptr) == L.LD_OK
    assert nnz[0] == Q.nnz and np.all(rp == -7)
    rp2, ci2, vv2 = mesh.spde_csr(p, t, 2.0, 2)
    assert np.array_equal(rp2, Q.indptr) and np.array_equal(ci2, Q.indices)
    assert np.abs(vv2 - Q.data).max() <= 1e-13 * np.abs(Q.data).max()


@pytest.mark.parametrize("alpha,d", [(1, 1), (1, 3), (2, 1), (2, 2)])
def test_mesh_colouring_and_bounds(lib, alpha, d):
    p, t = synth.perturbed_triangulation(11, 17, 21)
    Q = om.fem_spde_precision(p, t, 7.5, alpha)
    rp, ci, vv = om.csr_arrays(Q)
    col, nc = L.ld_colour_csr(rp, ci, d)
    assert np.array_equal(col, probing.colour_greedy(Q, d))
    assert probing.is_valid_colouring(Q, d, col)
    lo, hi = L.ld_csr_bounds(rp, ci, vv)
    ev = np.linalg.eigvalsh(Q.toarray())
    assert 0 < lo <= ev.min() and hi >= ev.max()
