"""The C ABI used from plain C: tests/c_client/momentum_box.c is compiled
against include/lbm.h and linked with liblbm.so and the CUDA runtime only,
then run; its conservation sums follow the exact momentum budget of a
periodic box under a uniform force."""
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1202_6081_gb300")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_1202_6081_gb300 import build
    build()
    exe = str(tmp_path_factory.mktemp("c_client") / "momentum_box")
    subprocess.run(["gcc", "-O2", "-std=c99", os.path.join(ROOT, "tests", "c_client",
                                                              "momentum_box.c"),
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
                    "-L", PKG, "-llbm", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
                    "-Wl,-rpath," + PKG, "-Wl,-rpath," + os.path.join(CUDA, "lib64"),
                    "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("dims", [(16, 16, 16, 100), (24, 10, 7, 37)])
def test_c_client_momentum_budget(client, dims):
    nx, ny, nz, steps = dims
    out = subprocess.run([client] + [str(v) for v in dims], capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    rows = np.array([[float(v) for v in line.split()] for line in out.stdout.split("\n")
                     if line.strip()])
    N = nx * ny * nz
    F = np.array([1e-5, -2e-5, 3e-5], dtype=np.float32).astype(np.float64)
    for t, mass, px, py, pz in rows:
        assert mass == pytest.approx(N, rel=1e-8)  # FP32 storage and per-cell values
        np.testing.assert_allclose([px, py, pz], N * F * t, rtol=1e-5, atol=1e-12 * N)
    assert rows[-1, 0] == 3 * steps
