"""Seeded random configurations against the FP64 oracle: lattice, grid
(including one-cell and odd extents), walls, uniform force or force field,
two-buffer or in-place streaming, graph run length and step count all
drawn at random, so that combinations no targeted test names are still
held to the oracle."""
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


def _config(i):
    rng = W.rng(9000 + i)
    Q = int(rng.choice([15, 27]))
    nx = int(rng.integers(1, 41))
    ny = int(rng.integers(1, 13))
    nz = int(rng.integers(1, 13))
    bc = int(rng.integers(0, 4))
    inplace = bool(nx % 2 == 0 and rng.integers(0, 2))
    field = bool(rng.integers(0, 2))
    steps = int(rng.integers(1, 12))
    graph_steps = int(rng.choice([0, 2, 4]))
    omega_nu = float(rng.uniform(0.8, 1.97))  # up to the tau = 0.51 end of the sweep
    return Q, (nz, ny, nx), bc, inplace, field, steps, graph_steps, omega_nu


@pytest.mark.parametrize("i", range(40))
def test_random_configuration_matches_oracle(lbm, orc, i):
    """omega_nu up to 1.97 (past the tau = 0.51 end of the bench's sweep),
    and every third configuration with all rates random in (0.3, 1.97)."""
    Q, shape, bc, inplace, field, steps, graph_steps, omega_nu = _config(i)
    rng = W.rng(9100 + i)
    if field:
        F = rng.uniform(-2e-4, 2e-4, (3,) + shape).astype(np.float32).astype(np.float64)
    else:
        F = rng.uniform(-2e-4, 2e-4, 3).astype(np.float32).astype(np.float64)
    rho = 1.0 + rng.uniform(-0.01, 0.01, shape)
    u = rng.uniform(-0.04, 0.04, (3,) + shape)
    f0 = orc.equilibrium(Q, rho, u, F) + rng.uniform(-1e-3, 1e-3, (Q,) + shape)
    om = W.omegas(Q, omega_nu)
    if i % 3 == 2:  # every rate drawn, distinct, up to 1.97
        om = W.random_omegas(Q, lo=0.3, hi=1.97, seed=9700 + i)
    S = lbm.Solver(Q, shape, om, force=F, walls=bc, inplace=inplace)
    S.set_graph_steps(graph_steps)
    S.set_state(f0)
    S.step(steps)
    torch.cuda.synchronize()
    got = S.get_state().cpu().numpy()
    want = orc.run(Q, shape, f0, F, om, steps, bc=bc)
    err = np.abs(got - want).max()
    assert err <= 3e-6, (Q, shape, bc, inplace, field, steps, graph_steps, omega_nu, err)


@pytest.mark.parametrize("i", range(32))
def test_random_adjoint_configuration_matches_oracle(lbm, orc, i):
    """The adjoint step (one-cell or two-cell kernel by the parity of nx) and
    the kinetic-energy seed on random grids, walls, storage types and forces,
    against the oracle's complex-step adjoint: D3Q27 for i < 20, D3Q15
    after."""
    rng = W.rng(9500 + i)
    Q = 27 if i < 20 else 15
    shape = (int(rng.integers(1, 9)), int(rng.integers(1, 9)), int(rng.integers(1, 25)))
    bc = int(rng.integers(0, 4))
    storage = str(rng.choice(["f32", "f16", "bf16"]))
    field = bool(rng.integers(0, 2))
    F = (rng.uniform(-1e-3, 1e-3, (3,) + shape) if field else rng.uniform(-1e-3, 1e-3, 3))
    F = F.astype(np.float32).astype(np.float64)
    rho = 1.0 + rng.uniform(-0.01, 0.01, shape)
    u = rng.uniform(-0.05, 0.05, (3,) + shape)
    om = W.random_omegas(Q, hi=1.97, seed=9600 + i)
    S = lbm.Solver(Q, shape, om, force=F, walls=bc, storage=storage)
    S.init_equilibrium(rho, u)
    f_t = S.get_state().cpu().numpy()  # the stored state, as the kernels read it
    lam_next = rng.standard_normal((Q,) + shape)
    ln = S.new_adjoint_field()
    S.adjoint_view(ln).copy_(torch.as_tensor(lam_next, dtype=torch.float32))
    lo = S.new_adjoint_field()
    gF = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    S.adjoint_step(S.current_buffer(), ln, lo, gF)
    seed = S.new_adjoint_field()
    S.kinetic_energy_seed(S.current_buffer(), seed)
    torch.cuda.synchronize()
    gF_want = np.zeros((3,) + shape)
    want = orc.adjoint_step(Q, shape, f_t, F, om, lam_next, bc=bc, gF=gF_want)
    got = S.adjoint_view(lo).cpu().numpy()
    cfg = (Q, shape, bc, storage, field)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max(), cfg
    assert np.abs(gF.cpu().numpy() - gF_want).max() <= 1e-5 * np.abs(gF_want).max(), cfg
    seed_want, _ = orc.kinetic_energy_grad(Q, f_t, F)
    assert np.abs(S.adjoint_view(seed).cpu().numpy() - seed_want).max() <= 1e-6, cfg
