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
    omega_nu = float(rng.uniform(0.8, 1.9))
    return Q, (nz, ny, nx), bc, inplace, field, steps, graph_steps, omega_nu


@pytest.mark.parametrize("i", range(40))
def test_random_configuration_matches_oracle(lbm, orc, i):
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
    S = lbm.Solver(Q, shape, om, force=F, walls=bc, inplace=inplace)
    S.set_graph_steps(graph_steps)
    S.set_state(f0)
    S.step(steps)
    torch.cuda.synchronize()
    got = S.get_state().cpu().numpy()
    want = orc.run(Q, shape, f0, F, om, steps, bc=bc)
    err = np.abs(got - want).max()
    assert err <= 3e-6, (Q, shape, bc, inplace, field, steps, graph_steps, omega_nu, err)
