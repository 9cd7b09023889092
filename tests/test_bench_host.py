"""Host-side logic of bench.py (no GPU): the general-mesh workload's spectral interval, the
algorithmic-byte accounting, and the guard that drops a recorded DRAM traffic figure once
the kernel sources it was captured from have changed."""
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import bench


def test_mesh_interval_encloses_the_spectrum():
    """The mesh line passes [lambda_min, lambda_max] to the library instead of estimating
    it: the lumped-mass lower bound and the row-sum upper bound must enclose the spectrum of
    the alpha = 2 FEM precision it builds (checked on a small mesh by shift-invert Lanczos)."""
    pytest.importorskip("paper_1105_5256_gb300")
    try:
        rp, ci, vv, lo, hi = bench.mesh_problem(40)
    except ImportError as e:   # the assembly needs the built library (host code only)
        pytest.skip(str(e))
    n = rp.size - 1
    Q = sp.csr_matrix((vv, ci, rp), shape=(n, n))
    lmin = spla.eigsh(Q.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    lmax = spla.eigsh(Q, k=1, which="LA", return_eigenvectors=False)[0]
    assert 0.0 < lo <= lmin and lmax <= hi


def test_algorithmic_bytes_follow_the_state_words():
    """4 state words a vertex and column per pass (r, p read and written), 2 more with the
    kept seed solution, plus the matrix's own bytes once a pass."""
    n, T, word, tile_iters = 1000, 4, 4, 30
    assert bench.algorithmic_bytes(n, T, word, tile_iters) == 4 * n * T * word * tile_iters
    assert bench.algorithmic_bytes(n, T, word, tile_iters, keep_x=True) == 6 * n * T * word * tile_iters
    assert (bench.algorithmic_bytes(n, T, word, tile_iters, bq_per_pass=123, passes=7)
            == 4 * n * T * word * tile_iters + 123 * 7)


def test_recorded_traffic_is_dropped_when_the_kernel_changes(tmp_path, monkeypatch):
    """A profile's traffic figure is used only while the sources it names hash to the
    recorded sha256."""
    csrc = tmp_path / "paper_1105_5256_gb300" / "csrc"
    csrc.mkdir(parents=True)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (csrc / "a.cuh").write_text("kernel one\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.pass_kernel_sha256(("a.cuh",))
    (prof / "p.md").write_text("engine_sources: a.cuh\nengine_sha256: %s\ntraffic_bytes_per_pass: 1234\n"
                               "traffic_bytes_per_vertex_tile_pass: 5.5\n" % sha)
    assert bench.recorded_traffic("p.md") == 1234.0
    assert bench.recorded_traffic("p.md", "traffic_bytes_per_vertex_tile_pass") == 5.5
    (csrc / "a.cuh").write_text("kernel two\n")
    assert bench.recorded_traffic("p.md") is None
    assert bench.recorded_traffic("missing.md") is None

