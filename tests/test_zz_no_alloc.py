"""lbm_conservation_noalloc: the conservation sums for callers that cannot
let the library allocate device memory (codes that plan all device memory
once from their own pool, or cannot afford the synchronisation an
allocation may imply).  It must give the same sums as lbm_conservation,
which allocates its scratch on first use, call after call, although every
call reuses one fixed array inside the library.

This file is collected last on purpose: it runs after every other test in a
full run, and also passes alone in a fresh process."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1202_6081_gb300 import build
    from paper_1202_6081_gb300 import lbm as mod
    build()
    mod.load()
    return mod


def _noalloc(lbm, S):
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    lbm.lbm_conservation_noalloc(S.ctx, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_conservation_on_two_calls_in_a_row(lbm):
    # first call: a larger grid (3072 rows), D3Q27 with a uniform force;
    # second call: a smaller grid (480 rows), D3Q15 with walls, so it reads
    # fewer partial records than the first call left in the shared array
    cases = [(27, (48, 64, 64), 0, (1e-5, -2e-5, 3e-6)),
             (15, (24, 20, 16), 3, (2e-5, 0.0, 0.0))]
    for Q, shape, walls, F in cases:
        S = lbm.Solver(Q, shape, W.omegas(Q, 1 / 0.6), force=F, walls=walls)
        rho, u = W.taylor_green(shape, u0=0.02, noise=1e-3)
        S.init_equilibrium(rho, u)
        S.step(7)
        got = _noalloc(lbm, S)
        want = S.conservation()
        N = int(np.prod(shape))
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got[0] + N, want[0], rtol=0, atol=1e-9 * N)
        np.testing.assert_allclose(got[1:], want[1:], rtol=0, atol=1e-9 * N)


def test_noalloc_rejects_grids_beyond_its_array(lbm):
    shape = (257, 256, 2)  # ny * nz = 65792 rows > 65536
    S = lbm.Solver(27, shape, W.omegas(27, 1.2))
    S.init_equilibrium(np.ones(shape), np.zeros((3,) + shape))
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as err:
        lbm.lbm_conservation_noalloc(S.ctx, out)
    assert err.value.status == 1  # LBM_EINVAL


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_noalloc_matches_conservation_for_16bit_storage(lbm, storage):
    shape = (12, 20, 34)
    S = lbm.Solver(27, shape, W.omegas(27, 1 / 0.6), force=(2e-5, 0.0, -1e-5), walls=1,
                   storage=storage)
    rho, u = W.taylor_green(shape, u0=0.02, noise=1e-3)
    S.init_equilibrium(rho, u)
    S.step(5)
    got = _noalloc(lbm, S)
    want = S.conservation()
    N = int(np.prod(shape))
    np.testing.assert_allclose(got[0] + N, want[0], rtol=0, atol=1e-9 * N)
    np.testing.assert_allclose(got[1:], want[1:], rtol=0, atol=1e-9 * N)


def test_noalloc_rejects_bad_arguments_before_any_launch(lbm):
    """Every rejection below returns before anything is enqueued: a NULL or
    misaligned output, a plain host array the GPU cannot write, a context
    with no buffers bound or no state set.  The output buffer is left as it
    was."""
    import ctypes
    lib = lbm.load()
    shape = (4, 6, 8)
    om = W.omegas(27, 1.2)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # created, nothing bound
    ctx = lbm.lbm_create(27, shape[2], shape[1], shape[0], om)
    out = torch.full((8,), 7.0, dtype=torch.float64, device="cuda")
    try:
        assert lib.lbm_conservation_noalloc(ctx, ctypes.c_void_p(out.data_ptr()), stream) == 3
    finally:
        lbm.lbm_destroy(ctx)
    S = lbm.Solver(27, shape, om)
    # bound, no state set
    assert lib.lbm_conservation_noalloc(S.ctx, ctypes.c_void_p(out.data_ptr()), stream) == 3
    S.init_equilibrium(np.ones(shape), np.zeros((3,) + shape))
    assert lib.lbm_conservation_noalloc(S.ctx, None, stream) == 1
    assert lib.lbm_conservation_noalloc(S.ctx, ctypes.c_void_p(out.data_ptr() + 4),
                                        stream) == 1
    host = (ctypes.c_double * 4)()  # pageable host memory: the GPU cannot write it
    assert lib.lbm_conservation_noalloc(S.ctx, ctypes.cast(host, ctypes.c_void_p),
                                        stream) == 1
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)
    assert list(host) == [0.0] * 4
    # the Python binding checks the tensor before calling the library
    with pytest.raises(ValueError):
        lbm.lbm_conservation_noalloc(S.ctx, torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError):
        lbm.lbm_conservation_noalloc(S.ctx, torch.zeros(4, dtype=torch.float32, device="cuda"))
    # and a valid call still works afterwards
    got = _noalloc(lbm, S)
    np.testing.assert_allclose(got, 0.0, atol=1e-9)


def test_noalloc_writes_mapped_host_memory(lbm):
    """Page-locked host memory mapped into the GPU's address space is a valid
    output: the reduction kernel writes it across the host link."""
    shape = (6, 10, 16)
    S = lbm.Solver(27, shape, W.omegas(27, 1 / 0.6), force=(1e-5, 0.0, 0.0))
    rho, u = W.taylor_green(shape, u0=0.02, noise=1e-3)
    S.init_equilibrium(rho, u)
    S.step(3)
    out = torch.full((4,), float("nan"), dtype=torch.float64).pin_memory()
    import ctypes
    lib = lbm.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.lbm_conservation_noalloc(S.ctx, ctypes.c_void_p(out.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    want = S.conservation()
    N = int(np.prod(shape))
    got = out.numpy()
    np.testing.assert_allclose(got[0] + N, want[0], rtol=0, atol=1e-9 * N)
    np.testing.assert_allclose(got[1:], want[1:], rtol=0, atol=1e-9 * N)


def test_noalloc_refuses_another_device_current(lbm):
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    shape = (4, 4, 4)
    S = lbm.Solver(27, shape, W.omegas(27, 1.2), device="cuda:0")
    S.init_equilibrium(np.ones(shape), np.zeros((3,) + shape))
    out = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    with torch.cuda.device(1):
        with pytest.raises(lbm.LBMError) as err:
            lbm.lbm_conservation_noalloc(S.ctx, out)
    assert err.value.status == 3  # LBM_ESTATE
