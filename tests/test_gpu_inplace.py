"""In-place single-buffer streaming (the AA access pattern) against the
two-buffer pull scheme and the FP64 oracle.

The in-place scheme runs the same collision on the same inputs, so after
any number of steps its state must equal the two-buffer state bit for bit,
in every storage type and with walls; both meet the oracle at the
two-buffer tolerances."""
import ctypes

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


def pair(lbm, Q, shape, om, storage="f32", walls=0, force=(0.0, 0.0, 0.0)):
    two = lbm.Solver(Q, shape, om, force=force, walls=walls, storage=storage)
    one = lbm.Solver(Q, shape, om, force=force, walls=walls, storage=storage, inplace=True)
    return two, one


def states(*solvers):
    torch.cuda.synchronize()
    return [S.get_state() for S in solvers]


GRIDS = [(3, 4, 2), (7, 3, 6), (9, 10, 38), (2, 33, 64)]  # (nz, ny, nx), nx even


@pytest.mark.parametrize("Q", [27, 15])
@pytest.mark.parametrize("bc", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", GRIDS)
@pytest.mark.parametrize("force", [(3e-3, -2e-3, 1e-3), (0.0, 0.0, 0.0)])
def test_inplace_equals_two_buffer_bitwise(lbm, Q, bc, shape, force):
    """Random state, uniform force (or zero: the D3Q15 force-free kernels),
    random rates: after 1, 2, 3 and 6 steps (both parities of the in-place
    layout) the states are identical."""
    f0 = W.random_field_state(shape, Q, seed=300 + bc, spread=0.5)
    om = W.random_omegas(Q, seed=6)
    two, one = pair(lbm, Q, shape, om, walls=bc, force=force)
    two.set_state(f0)
    one.set_state(f0)
    done = 0
    for n in (1, 1, 1, 3):
        two.step(n)
        one.step(n)
        done += n
        a, b = states(two, one)
        assert torch.equal(a, b), (done, float((a - b).abs().max()))


@pytest.mark.parametrize("Q", [27, 15])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("force", [(1e-4, 0.0, -1e-4), (0.0, 0.0, 0.0)])
def test_inplace_16bit_storage_equals_two_buffer(lbm, Q, storage, force):
    shape = (6, 9, 20)
    rho, u = W.taylor_green(shape, u0=0.05, noise=1e-2, seed=41)
    om = W.omegas(Q, 1 / 0.6)
    two, one = pair(lbm, Q, shape, om, storage=storage, walls=3, force=force)
    two.init_equilibrium(rho, u)
    one.init_equilibrium(rho, u)
    for n in (1, 4):
        two.step(n)
        one.step(n)
        a, b = states(two, one)
        assert torch.equal(a, b)


@pytest.mark.parametrize("Q", [27, 15])
def test_inplace_force_field_and_readouts(lbm, Q):
    """Per-cell force field; macroscopic fields, conservation sums (both
    entry points) and the kinetic energy read the swapped layout correctly."""
    shape = (5, 12, 14)
    rho, u = W.taylor_green(shape, u0=0.05, noise=1e-2, seed=43)
    F = torch.as_tensor(W.rng(44).uniform(-1e-3, 1e-3, (3,) + shape), dtype=torch.float32,
                        device="cuda").contiguous()
    om = W.random_omegas(Q, seed=45)
    two, one = pair(lbm, Q, shape, om, walls=1)
    for S in (two, one):
        S.set_force_field(F)
        S.init_equilibrium(rho, u)
        S.step(3)  # odd: the in-place state is in its swapped layout
    torch.cuda.synchronize()
    r2, u2 = two.macroscopic()
    r1, u1 = one.macroscopic()
    assert torch.equal(r2, r1) and torch.equal(u2, u1)
    assert np.array_equal(two.conservation(), one.conservation())
    out2 = torch.empty(4, dtype=torch.float64, device="cuda")
    out1 = torch.empty(4, dtype=torch.float64, device="cuda")
    lbm.lbm_conservation_noalloc(two.ctx, out2)
    lbm.lbm_conservation_noalloc(one.ctx, out1)
    torch.cuda.synchronize()
    assert torch.equal(out2, out1)
    assert two.kinetic_energy() == one.kinetic_energy()


@pytest.mark.parametrize("Q", [27, 15])
def test_inplace_matches_oracle(lbm, orc, Q):
    """Walled channel with a force field, 5 steps, against the FP64 oracle
    (same bound as the two-buffer kernels)."""
    shape = (9, 10, 14)
    f0 = W.random_field_state(shape, Q, seed=47, spread=0.5)
    om = W.random_omegas(Q, seed=48)
    F = np.asarray(W.rng(49).uniform(-2e-3, 2e-3, (3,) + shape), dtype=np.float32)
    S = lbm.Solver(Q, shape, om, force=F, walls=3, inplace=True)
    S.set_state(f0)
    S.step(5)
    torch.cuda.synchronize()
    got = S.get_state().cpu().numpy()
    want = orc.run(Q, shape, f0, F.astype(np.float64), om, 5, bc=3)
    assert np.abs(got - want).max() <= 1e-5


def test_inplace_256cubed_equals_two_buffer(lbm):
    """The bench workload (D3Q27, 256^3 periodic, Taylor-Green + noise,
    tau = 0.6) in the launch configuration the bench times: after 10 and 11
    steps the in-place state equals the two-buffer state bit for bit."""
    Q, n = 27, 256
    shape = (n, n, n)
    rho, u = W.taylor_green(shape, u0=0.02, noise=1e-3)
    om = W.omegas(Q, 1 / 0.6)
    two, one = pair(lbm, Q, shape, om)
    two.init_equilibrium(rho, u)
    one.init_equilibrium(rho, u)
    for k in (10, 1):
        two.step(k)
        one.step(k)
        a, b = states(two, one)
        assert torch.equal(a, b)
        del a, b


def test_inplace_api_contract(lbm):
    """One buffer only; the calls that take two-buffer states are refused
    with LBM_EUNSUPPORTED, not run on the wrong layout."""
    lib = lbm.load()
    Q = 27
    om = W.omegas(Q, 1.2)
    ctx = lbm.lbm_create(Q, 6, 5, 4, om, bc_flags=lbm.LBM_INPLACE)
    try:
        a = torch.empty(lbm.lbm_state_bytes(ctx), dtype=torch.uint8, device="cuda")
        b = torch.empty_like(a)
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        assert lib.lbm_bind(ctx, p(a), p(b), None) == 1        # two buffers: EINVAL
        assert lib.lbm_bind(ctx, p(a), None, None) == 0
        assert lib.lbm_step(ctx, 1, None) == 3                 # no state yet
        lbm.lbm_init_equilibrium(ctx, torch.ones((4, 5, 6), dtype=torch.float64, device="cuda"),
                                 torch.zeros((3, 4, 5, 6), dtype=torch.float64, device="cuda"))
        assert lib.lbm_step(ctx, 3, None) == 0
        assert lib.lbm_current_state(ctx) is None
        assert lib.lbm_step_into(ctx, p(a), p(b), None) == 6   # LBM_EUNSUPPORTED
        lam = torch.zeros(lbm.lbm_adjoint_bytes(ctx) // 4, dtype=torch.float32, device="cuda")
        lam2 = torch.zeros_like(lam)
        assert lib.lbm_adjoint_step(ctx, p(a), p(lam), p(lam2), None, None) == 6
        assert lbm.lbm_conservation(ctx)[0] == pytest.approx(120.0, rel=1e-12)
    finally:
        torch.cuda.synchronize()
        lbm.lbm_destroy(ctx)
