"""Runs of steps launched as CUDA graphs give the same states, bit for bit,
as one launch per step, in both streaming schemes, and follow changes of
the force, rates and force field between calls."""
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


@pytest.mark.parametrize("Q", [27, 15])
@pytest.mark.parametrize("inplace", [False, True])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_graph_runs_equal_single_launches(lbm, Q, inplace, storage):
    shape = (6, 10, 16)
    rho, u = W.taylor_green(shape, u0=0.04, noise=1e-2, seed=61)
    om = W.random_omegas(Q, seed=62)
    F = torch.as_tensor(W.rng(63).uniform(-1e-3, 1e-3, (3,) + shape), dtype=torch.float32,
                        device="cuda").contiguous()
    runs = []
    for graph_steps in (0, 4):
        S = lbm.Solver(Q, shape, om, force=(1e-4, 0.0, -2e-4), walls=lbm.LBM_WALL_Y,
                       storage=storage, inplace=inplace)
        S.set_graph_steps(graph_steps)
        S.init_equilibrium(rho, u)
        S.step(13)                      # three graphs from parity 0, one single step
        S.step(9)                       # two graphs from parity 1, one single step
        S.set_force((3e-4, 1e-4, 0.0))  # a new force: a new graph
        S.step(8)
        S.set_omega(W.random_omegas(Q, seed=64))
        S.step(5)
        S.set_force_field(F)
        S.step(10)
        torch.cuda.synchronize()
        runs.append(S.get_state())
    assert torch.equal(runs[0], runs[1])


def test_graph_steps_argument_checks(lbm):
    lib = lbm.load()
    ctx = lbm.lbm_create(27, 8, 4, 4, W.omegas(27, 1.2))
    try:
        assert lib.lbm_set_graph_steps(ctx, 3) == 1   # odd: EINVAL
        assert lib.lbm_set_graph_steps(ctx, -2) == 1
        assert lib.lbm_set_graph_steps(ctx, 0) == 0
        assert lib.lbm_set_graph_steps(ctx, 64) == 0
    finally:
        lbm.lbm_destroy(ctx)


def test_steps_inside_a_callers_graph_capture(lbm):
    """lbm_step called while the caller captures its stream into a CUDA
    graph (torch.cuda.graph): the library sees the capture and launches each
    step on its own, so the caller's graph holds the steps; replaying it
    advances the state exactly like direct calls."""
    Q = 27
    shape = (4, 6, 10)
    rho, u = W.taylor_green(shape, u0=0.03, noise=1e-2, seed=71)
    om = W.omegas(Q, 1.4)
    ref = lbm.Solver(Q, shape, om, force=(1e-4, 0.0, 0.0))
    cap = lbm.Solver(Q, shape, om, force=(1e-4, 0.0, 0.0))
    ref.init_equilibrium(rho, u)
    cap.init_equilibrium(rho, u)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            cap.step(4, stream=s)  # an even count: the captured run returns to its parity
    torch.cuda.synchronize()
    for _ in range(5):
        g.replay()
    ref.step(20)
    torch.cuda.synchronize()
    assert torch.equal(ref.get_state(), cap.get_state())
