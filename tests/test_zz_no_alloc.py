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
