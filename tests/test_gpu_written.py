"""Every output element is written: the output buffers are filled with NaN
(all-ones bytes, a NaN in FP32, FP16 and BF16) before a call, and after it
no NaN may remain where the call's contract says it writes -- the
populations of every cell for a step and for an adjoint step, the adjoint
seeds, and the macroscopic fields.  An index that misses a cell or a
population would leave NaN behind; the step's values are also held to the
oracle, so a cell written twice with the wrong value fails too.  Both
lattices, all storage types, walls or none, both kernels (nx even: two
cells per thread; odd: one), no force or a force field."""
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


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def poison(t):
    t.view(torch.uint8).fill_(0xFF)
    return t


CASES = [(Q, storage, bc, shape, field)
         for Q in (27, 15)
         for storage in ("f32", "f16", "bf16")
         for bc in (0, 3)
         for shape in ((5, 6, 10), (5, 6, 9))
         for field in (False, True)]


@pytest.mark.parametrize("Q,storage,bc,shape,field", CASES)
def test_step_and_adjoint_write_every_element(lbm, orc, Q, storage, bc, shape, field):
    rng = W.rng(700 + Q + bc)
    om = W.random_omegas(Q, seed=701)
    if field:
        F = rng.uniform(-1e-3, 1e-3, (3,) + shape).astype(np.float32).astype(np.float64)
    else:
        F = np.zeros(3)
    rho, u = W.taylor_green(shape, u0=0.04, noise=1e-2, seed=702)
    S = lbm.Solver(Q, shape, om, force=F, walls=bc, storage=storage)
    S.init_equilibrium(rho, u)
    f_t = S.get_state().cpu().numpy()  # the stored state, as the kernels read it
    src = S.current_buffer()
    orig = src.clone()

    # one step into a poisoned buffer
    dst = poison(S.new_state_buffer())
    S.step_into(src, dst)
    S.load_buffer(dst)  # the new state becomes the current one (in src)
    got = S.get_state().cpu().numpy()
    assert np.isfinite(got).all(), "step left unwritten populations"
    want = orc.run(Q, shape, f_t, F, om, 1, bc=bc)
    # FP32 storage to FP32 rounding; 16-bit storage to one unit in the last
    # place of the stored deviation (f - w)/w times its weight, below 2e-4
    # here (|dev| < 0.3, BF16 ulp 2^-7 of its binade)
    tol = 2e-6 if storage == "f32" else 6e-4
    assert np.abs(got - want).max() <= tol

    # the macroscopic fields of the new state
    rho_out = poison(torch.empty(shape, dtype=torch.float32, device="cuda"))
    u_out = poison(torch.empty((3,) + shape, dtype=torch.float32, device="cuda"))
    lbm.lbm_macroscopic(S.ctx, rho_out, u_out, None)
    torch.cuda.synchronize()
    assert torch.isfinite(rho_out).all() and torch.isfinite(u_out).all()

    # one adjoint step from the original state into a poisoned adjoint field
    S.load_buffer(orig)
    ln = S.new_adjoint_field()
    S.adjoint_view(ln).copy_(torch.as_tensor(rng.standard_normal((Q,) + shape),
                                             dtype=torch.float32))
    lo = poison(S.new_adjoint_field())
    gF = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    S.adjoint_step(src, ln, lo, gF)
    torch.cuda.synchronize()
    assert torch.isfinite(S.adjoint_view(lo)).all(), "adjoint left unwritten elements"
    assert torch.isfinite(gF).all()

    # the seeds into poisoned adjoint fields
    for seed in ("energy", "macro"):
        lam = poison(S.new_adjoint_field())
        if seed == "energy":
            S.kinetic_energy_seed(src, lam)
        else:
            g_u = torch.ones((3,) + shape, dtype=torch.float32, device="cuda")
            S.macroscopic_seed(src, None, g_u, lam)
        torch.cuda.synchronize()
        assert torch.isfinite(S.adjoint_view(lam)).all(), seed
