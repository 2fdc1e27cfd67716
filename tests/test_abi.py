"""The C-ABI library builds, loads and exports every entry point that
include/lbm.h declares; argument validation needs no GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1202_6081_gb300 import build, lbm
    build()
    return lbm.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("lbm_create", "lbm_step", "lbm_macroscopic", "lbm_conservation", "lbm_destroy"):
        assert n in names


def test_every_declared_function_is_exported(lib):
    so = os.path.join(ROOT, "paper_1202_6081_gb300", "liblbm.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(lbm_[a-z_0-9]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        getattr(lib, n)


def _om(Q, v=1.5):
    return (ctypes.c_double * Q)(*([0.0] * 4 + [v] * (Q - 4)))


@pytest.mark.parametrize("args", [
    dict(lattice=19), dict(nx=0), dict(ny=-1), dict(nz=0), dict(bc=16), dict(storage=3),
    dict(bc=4, nx=5), dict(bc=7, nx=7),  # in-place streaming takes cell pairs: nx even
    dict(nx=2048, ny=1024, nz=1024),      # 2^31 cells: beyond 32-bit plane offsets
    dict(nx=1, ny=65536, nz=1),           # launch grid limit in y
    dict(omega_value=2.0), dict(omega_value=0.0), dict(omega_value=float("nan")),
    dict(force=(float("inf"), 0.0, 0.0)), dict(omega_null=True), dict(out_null=True),
    dict(bc=8, storage=1), dict(bc=8, storage=2),  # stochastic FP32 update: FP32 storage only
    dict(bc=12, nx=6),                             # and not in place
])
def test_create_rejects_bad_arguments_before_touching_cuda(lib, args):
    Q = args.get("lattice", 27)
    om = None if args.get("omega_null") else _om(Q if Q in (15, 27) else 27,
                                                args.get("omega_value", 1.5))
    F = (ctypes.c_double * 3)(*args["force"]) if "force" in args else None
    ctx = ctypes.c_void_p()
    out = None if args.get("out_null") else ctypes.byref(ctx)
    st = lib.lbm_create(Q, args.get("nx", 4), args.get("ny", 4), args.get("nz", 4), om, F,
                        args.get("bc", 0), args.get("storage", 0), out)
    assert st == 1  # LBM_EINVAL
    assert not ctx.value


def test_null_context_calls_are_safe(lib):
    lib.lbm_destroy(None)
    assert lib.lbm_state_bytes(None) == 0
    assert lib.lbm_step(None, 1, None) == 1
    assert lib.lbm_conservation(None, None, None) == 1
    assert lib.lbm_status_string(0).decode() == "LBM_OK"
    assert "EINVAL" in lib.lbm_status_string(1).decode()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without liblbm.so the binding raises instead of
    computing anything another way."""
    from paper_1202_6081_gb300 import lbm
    monkeypatch.setattr(lbm, "_lib", None)
    monkeypatch.setattr(lbm, "LIB_PATH", str(tmp_path / "liblbm.so"))
    with pytest.raises(RuntimeError, match="liblbm.so not found"):
        lbm.load()
    with pytest.raises(RuntimeError):
        lbm.lbm_create(27, 4, 4, 4, [1.0] * 27)


def test_no_gpu_fails_loudly(lib):
    """Without a usable GPU, creating a context reports LBM_ECUDA (or the
    Solver raises before that); nothing runs on the CPU instead."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1202_6081_gb300 import lbm
    with pytest.raises(Exception):
        lbm.lbm_create(27, 4, 4, 4, [1.0] * 27)
    with pytest.raises(Exception):
        lbm.Solver(27, (4, 4, 4), [1.0] * 27)
