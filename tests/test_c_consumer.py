"""The boundary from C (no GPU): tests/c_consumer.c includes include/logdet.h as C99 with
warnings as errors, links liblogdet.so and calls the host-only entry points (colouring,
quadrature nodes, the CSR spectral interval, finite-element assembly, error reporting)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1105_5256_gb300 import _build
    return _build.build()


def test_header_compiles_as_c99_and_host_calls_work(libpath, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    exe = tmp_path / "c_consumer"
    libdir = os.path.dirname(libpath)
    cmd = ["gcc", "-std=c99", "-D_DEFAULT_SOURCE", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_consumer.c"),
           "-o", str(exe), "-L", libdir, "-l:liblogdet.so", "-Wl,-rpath," + libdir, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith("ok ")
    fields = dict(kv.split("=") for kv in r.stdout.split()[1:])
    # 4 diagonal entries + both directions of the 5 edges, less the zero coupling across
    # the shared hypotenuse (its opposite angles are right angles) in both directions
    assert int(fields["nnz"]) == 12
    assert abs(float(fields["total"]) - 1.0) < 1e-14
