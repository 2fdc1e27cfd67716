"""The discrete adjoint on the GPU (through the C ABI), D3Q27 and D3Q15,
against the FP64 oracle's adjoint (complex-step Jacobians), against FP64 central finite
differences of the oracle, and, at the 128^3 workload, against central
finite differences of the GPU forward.

J(F) = sum_x rho |u|^2 / 2 after n steps from a fixed initial state, as a
function of the per-cell force field F used by the steps."""
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


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def to_pitched(S, dense):
    lam = S.new_adjoint_field()
    S.adjoint_view(lam).copy_(torch.as_tensor(dense, dtype=torch.float32))
    return lam


@pytest.mark.parametrize("Q", [27, 15])
@pytest.mark.parametrize("bc", [0, 3])
@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("shape", [(6, 7, 10), (6, 7, 9)])  # two-cell and one-cell kernels
def test_adjoint_step_matches_oracle(lbm, orc, Q, bc, storage, shape):
    rho, u = W.taylor_green(shape, u0=0.05, noise=1e-2, seed=31)
    om = W.random_omegas(Q, seed=32)
    F = f32(W.rng(33).uniform(-1e-3, 1e-3, (3,) + shape))
    lam_next = W.rng(34).standard_normal((Q,) + shape)
    S = lbm.Solver(Q, shape, om, force=F, walls=bc, storage=storage)
    S.init_equilibrium(rho, u)
    f_t = S.current_buffer()
    f_stored = S.get_state().cpu().numpy()
    ln = to_pitched(S, lam_next)
    lo = S.new_adjoint_field()
    gF = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    S.adjoint_step(f_t, ln, lo, gF)
    torch.cuda.synchronize()
    got = S.adjoint_view(lo).cpu().numpy()
    gF_want = np.zeros((3,) + shape)
    want = orc.adjoint_step(Q, shape, f_stored, F, om, lam_next, bc=bc, gF=gF_want)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    assert np.abs(gF.cpu().numpy() - gF_want).max() <= 1e-5 * np.abs(gF_want).max()


@pytest.mark.parametrize("Q", [27, 15])
def test_kinetic_energy_and_seed_match_oracle(lbm, orc, Q):
    shape = (5, 8, 12)
    rho, u = W.taylor_green(shape, u0=0.05, noise=1e-2, seed=35)
    F = f32(W.rng(36).uniform(-1e-3, 1e-3, (3,) + shape))
    S = lbm.Solver(Q, shape, W.omegas(Q, 1.4), force=F, walls=1)
    S.init_equilibrium(rho, u)
    f = S.get_state().cpu().numpy()
    J = S.kinetic_energy()
    assert J == pytest.approx(orc.kinetic_energy(Q, f, F), rel=1e-6)
    lam = S.new_adjoint_field()
    gF = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    S.kinetic_energy_seed(S.current_buffer(), lam, gF)
    dfl, dF = orc.kinetic_energy_grad(Q, f, F)
    np.testing.assert_allclose(S.adjoint_view(lam).cpu().numpy(), dfl, atol=1e-7)
    np.testing.assert_allclose(gF.cpu().numpy(), dF, atol=1e-8)


def _cells(shape, k, seed):
    cells = W.sample_cells(shape, k, seed=seed)
    comps = W.rng(seed + 1).integers(0, 3, size=len(cells))
    return [(int(c), tuple(int(v) for v in np.unravel_index(c, shape))) for c in cells], comps


def test_gradient_matches_fp64_finite_differences(lbm, orc):
    """16^3 periodic, Taylor-Green + noise, Gaussian force field (RMS 1e-5),
    200 steps, checkpoint every 20: the GPU adjoint gradient matches FP64
    central differences of the oracle (eps = 1e-6) on 16 sampled
    (cell, component) pairs, each within 1e-3 of its own value."""
    from paper_1202_6081_gb300.autograd import kinetic_energy_after
    Q = 27
    shape = (16, 16, 16)
    om = W.omegas(Q, 1 / 0.6)
    rho, u = W.taylor_green(shape, u0=0.02, noise=1e-3)
    F0 = f32(W.gaussian_force_field(shape, rms=1e-5, sigma=4.0))
    S = lbm.Solver(Q, shape, om)
    Ft = torch.as_tensor(F0, dtype=torch.float32, device="cuda").contiguous().requires_grad_()
    S.set_force_field(Ft.detach())
    S.init_equilibrium(rho, u)
    f0 = orc.equilibrium(Q, rho, u, F0)  # fixed initial state of the FD runs
    J = kinetic_energy_after(S, Ft, 200, 20)
    J.backward()
    g = Ft.grad.cpu().numpy()
    samples, comps = _cells(shape, 16, seed=41)
    eps = 1e-6
    fd = []
    for (c, (z, y, x)), k in zip(samples, comps):
        Fp = F0.copy()
        Fp[k, z, y, x] += eps
        Fm = F0.copy()
        Fm[k, z, y, x] -= eps
        jp = orc.kinetic_energy(Q, orc.run(Q, shape, f0, Fp, om, 200), Fp)
        jm = orc.kinetic_energy(Q, orc.run(Q, shape, f0, Fm, om, 200), Fm)
        fd.append((jp - jm) / (2 * eps))
    fd = np.array(fd)
    got = np.array([g[k, z, y, x] for (c, (z, y, x)), k in zip(samples, comps)])
    print("fd", fd[:4], "adjoint", got[:4])
    assert_per_element(got, fd)


def assert_per_element(got, fd, rel=1e-3, floor=1e-5):
    """Every sampled derivative on its own: |got - fd| <= rel |fd| plus a
    small floor relative to the largest sampled derivative (for entries
    near zero)."""
    err = np.abs(got - fd)
    bound = rel * np.abs(fd) + floor * np.abs(fd).max()
    print("per-element |adjoint - fd| / |fd|:", np.array2string(err / np.abs(fd), precision=2))
    assert np.all(err <= bound), (got, fd)


def test_gradient_32cubed_matches_fp64_oracle_differences(lbm, orc):
    """The adjoint workload's recipe at 32^3: D3Q27 periodic, tau = 0.6,
    Taylor-Green + noise, Gaussian force field (RMS 1e-5, sigma 4), J after
    200 steps, checkpoint every 20.  The GPU gradient against FP64 central
    differences of the oracle on 16 (cell, component) pairs, each within
    1e-3 of its own value (plus a 1e-5 floor of the largest).  The step
    eps = 1e-8 (1e-3 of the force's RMS) lies on a plateau: on four of the
    pairs the difference quotient at eps = 1e-7 agrees to 1e-4 (measured
    ~1e-7; at 1e-9 FP64 roundoff starts to show, ~4e-7)."""
    from paper_1202_6081_gb300.autograd import kinetic_energy_after
    Q = 27
    shape = (32, 32, 32)
    om = W.omegas(Q, 1 / 0.6)
    rho, u = W.taylor_green(shape, u0=0.02, noise=1e-3)
    F0 = f32(W.gaussian_force_field(shape, rms=1e-5, sigma=4.0))
    S = lbm.Solver(Q, shape, om)
    Ft = torch.as_tensor(F0, dtype=torch.float32, device="cuda").contiguous().requires_grad_()
    S.set_force_field(Ft.detach())
    S.init_equilibrium(rho, u)
    f0 = orc.equilibrium(Q, rho, u, F0)
    J = kinetic_energy_after(S, Ft, 200, 20)
    J.backward()
    g = Ft.grad.cpu().numpy()
    cells = W.sample_cells(shape, 16, seed=43)
    comps = W.rng(44).integers(0, 3, size=len(cells))

    def quotient(z, y, x, k, eps):
        Fp, Fm = F0.copy(), F0.copy()
        Fp[k, z, y, x] += eps
        Fm[k, z, y, x] -= eps
        jp = orc.kinetic_energy(Q, orc.run(Q, shape, f0, Fp, om, 200), Fp)
        jm = orc.kinetic_energy(Q, orc.run(Q, shape, f0, Fm, om, 200), Fm)
        return (jp - jm) / (2 * eps)

    fd, got = [], []
    for n, (c, k) in enumerate(zip(cells, comps)):
        z, y, x = (int(v) for v in np.unravel_index(c, shape))
        q8 = quotient(z, y, x, k, 1e-8)
        if n < 4:
            q7 = quotient(z, y, x, k, 1e-7)
            assert abs(q7 - q8) <= 1e-4 * abs(q8), (q7, q8)
        fd.append(q8)
        got.append(g[k, z, y, x])
    fd, got = np.array(fd), np.array(got)
    print("fd", fd[:4], "adjoint", got[:4])
    assert_per_element(got, fd)


def test_gradient_128cubed_matches_gpu_finite_differences(lbm):
    """The adjoint workload itself: D3Q27, 128^3 periodic, tau = 0.6,
    Taylor-Green + noise, Gaussian force field RMS 1e-5, J after 200 steps,
    checkpoint every 20.  A check that the workload runs end to end: the
    gradient matches central differences of the GPU's own FP32 forward on 16
    random cells to 5e-3 relative to the largest sampled gradient.  Those
    differences carry FP32 noise of about 1e-3 of the largest (measured
    1.0e-3 and 1.3e-3 in two builds whose forward steps round differently);
    the check against the FP64 definition is the 32^3 test above."""
    from paper_1202_6081_gb300.autograd import kinetic_energy_after
    Q = 27
    shape = (128, 128, 128)
    om = W.omegas(Q, 1 / 0.6)
    rho, u = W.taylor_green(shape, u0=0.02, noise=1e-3)
    F0 = W.gaussian_force_field(shape, rms=1e-5, sigma=4.0).astype(np.float32)
    S = lbm.Solver(Q, shape, om)
    Ft = torch.as_tensor(F0, device="cuda").contiguous().requires_grad_()
    S.set_force_field(Ft.detach())
    S.init_equilibrium(rho, u)
    init = S.current_buffer().clone()
    J = kinetic_energy_after(S, Ft, 200, 20)
    J.backward()
    g = Ft.grad

    def J_of(Fdev):
        S.set_force_field(Fdev)
        S.load_buffer(init)
        S.step(200)
        return S.kinetic_energy()

    samples, comps = _cells(shape, 16, seed=42)
    eps = 4e-5
    fd, got = [], []
    Fp = Ft.detach().clone()
    for (c, (z, y, x)), k in zip(samples, comps):
        base = float(Fp[k, z, y, x])
        Fp[k, z, y, x] = base + eps
        hi = float(Fp[k, z, y, x])
        jp = J_of(Fp)
        Fp[k, z, y, x] = base - eps
        lo = float(Fp[k, z, y, x])
        jm = J_of(Fp)
        Fp[k, z, y, x] = base
        fd.append((jp - jm) / (hi - lo))
        got.append(float(g[k, z, y, x]))
    fd, got = np.array(fd), np.array(got)
    print("fd", fd[:4], "adjoint", got[:4], "max error / max |fd| = %.2e"
          % (np.abs(got - fd).max() / np.abs(fd).max()))
    assert np.abs(got - fd).max() <= 5e-3 * np.abs(fd).max()


@pytest.mark.parametrize("Q", [27, 15])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_macroscopic_seed_matches_oracle(lbm, orc, Q, storage):
    """Seed of the adjoint for an objective J(rho, u): lam = dJ/df and the
    direct dJ/dF against the oracle's chain rule, walled grid, force field."""
    shape = (5, 7, 10)
    rho, u = W.taylor_green(shape, u0=0.05, noise=1e-2, seed=51)
    F = f32(W.rng(52).uniform(-1e-3, 1e-3, (3,) + shape))
    g_rho = f32(W.rng(53).standard_normal(shape))
    g_u = f32(W.rng(54).standard_normal((3,) + shape))
    S = lbm.Solver(Q, shape, W.omegas(Q, 1.3), force=F, walls=3, storage=storage)
    S.init_equilibrium(rho, u)
    f = S.get_state().cpu().numpy()
    lam = S.new_adjoint_field()
    gF = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    S.macroscopic_seed(S.current_buffer(), torch.as_tensor(g_rho, dtype=torch.float32),
                       torch.as_tensor(g_u, dtype=torch.float32), lam, gF)
    torch.cuda.synchronize()
    want, want_F = orc.macroscopic_grad(Q, f, F, g_rho, g_u)
    got = S.adjoint_view(lam).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    assert np.abs(gF.cpu().numpy() - want_F).max() <= 1e-5 * np.abs(want_F).max()
    # a missing gradient counts as zero
    S.macroscopic_seed(S.current_buffer(), None, torch.as_tensor(g_u, dtype=torch.float32), lam)
    torch.cuda.synchronize()
    want0, _ = orc.macroscopic_grad(Q, f, F, 0.0, g_u)
    assert np.abs(S.adjoint_view(lam).cpu().numpy() - want0).max() <= 1e-5 * np.abs(want0).max()


@pytest.mark.parametrize("Q", [27, 15])
def test_macroscopic_after_gradients_match_fp64_differences(lbm, orc, Q):
    """A torch objective of the final (rho, u), J = <c, u> + <d, rho^2>, back-
    propagated through 30 steps (checkpoints every 7, so the last segment is
    short) on a walled 6 x 8 x 10 grid: dJ/dF and dJ/df0 match FP64 central
    differences of the oracle on 12 sampled entries each."""
    from paper_1202_6081_gb300.autograd import macroscopic_after
    shape = (6, 8, 10)
    om = W.omegas(Q, 1 / 0.7)
    rho0, u0 = W.taylor_green(shape, u0=0.03, noise=2e-3, seed=55)
    F0 = f32(W.rng(56).uniform(-1e-4, 1e-4, (3,) + shape))
    f0 = orc.equilibrium(Q, rho0, u0, F0)
    c = torch.as_tensor(W.rng(57).standard_normal((3,) + shape), dtype=torch.float32,
                        device="cuda")
    d = torch.as_tensor(W.rng(58).standard_normal(shape), dtype=torch.float32, device="cuda")
    S = lbm.Solver(Q, shape, om, walls=3)
    Ft = torch.as_tensor(F0, dtype=torch.float32, device="cuda").contiguous().requires_grad_()
    f0t = torch.as_tensor(f0, device="cuda").requires_grad_()
    rho, u = macroscopic_after(S, Ft, 30, every=7, f0=f0t)
    J = (c * u).sum() + (d * rho * rho).sum()
    J.backward()
    gF, gf0 = Ft.grad.cpu().numpy(), f0t.grad.cpu().numpy()
    cn, dn = c.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64)

    def J_or(f_init, F):
        r, v = orc.macroscopic(Q, orc.run(Q, shape, f_init, F, om, 30, bc=3), F)
        return np.sum(cn * v) + np.sum(dn * r * r)

    rng = W.rng(59)
    eps = 1e-6
    fdF, gotF, fdf, gotf = [], [], [], []
    for _ in range(12):
        k, z, y, x = (int(rng.integers(0, n)) for n in (3,) + shape)
        Fp, Fm = F0.copy(), F0.copy()
        Fp[k, z, y, x] += eps
        Fm[k, z, y, x] -= eps
        fdF.append((J_or(f0, Fp) - J_or(f0, Fm)) / (2 * eps))
        gotF.append(gF[k, z, y, x])
        a = int(rng.integers(0, Q))
        fp, fm = f0.copy(), f0.copy()
        fp[a, z, y, x] += eps
        fm[a, z, y, x] -= eps
        fdf.append((J_or(fp, F0) - J_or(fm, F0)) / (2 * eps))
        gotf.append(gf0[a, z, y, x])
    fdF, gotF, fdf, gotf = map(np.array, (fdF, gotF, fdf, gotf))
    print("dJ/dF fd", fdF[:3], "adjoint", gotF[:3], "; dJ/df0 fd", fdf[:3], "adjoint", gotf[:3])
    assert_per_element(gotF, fdF)
    assert_per_element(gotf, fdf)


@pytest.mark.parametrize("Q", [27, 15])
def test_adjoint_entry_points_reject_bad_arguments(lbm, Q):
    """The adjoint calls check their pointers before launching anything:
    misaligned or aliased adjoint fields, a misaligned dJ/dF, a state buffer
    off its 256-byte alignment, overlapping state buffers for lbm_step_into
    and a seed before any state are LBM_EINVAL / LBM_ESTATE; the same call
    with good arguments succeeds."""
    import ctypes
    lib = lbm.load()
    shape = (4, 5, 6)
    ctx = lbm.lbm_create(Q, shape[2], shape[1], shape[0], W.omegas(Q, 1.2))
    try:
        nb = lbm.lbm_state_bytes(ctx)
        a = torch.empty(nb, dtype=torch.uint8, device="cuda")
        b = torch.empty_like(a)
        p = lambda t, off=0: ctypes.c_void_p(t.data_ptr() + off)
        lam = torch.zeros(lbm.lbm_adjoint_bytes(ctx) // 4 + 4, dtype=torch.float32, device="cuda")
        lam2 = torch.zeros_like(lam)
        gF = torch.zeros(3 * 120 + 1, dtype=torch.float32, device="cuda")
        seed = lib.lbm_kinetic_energy_seed
        msd = lib.lbm_macroscopic_seed
        assert seed(ctx, None, p(lam), None, None) == 3             # no state bound yet
        assert msd(ctx, None, None, None, p(lam), None, None) == 3
        assert lib.lbm_bind(ctx, p(a), p(b), None) == 0
        lbm.lbm_init_equilibrium(ctx, torch.ones(shape, dtype=torch.float64, device="cuda"),
                                 torch.zeros((3,) + shape, dtype=torch.float64, device="cuda"))
        step = lib.lbm_adjoint_step
        assert step(ctx, p(a), p(lam), p(lam), None, None) == 1       # aliased fields
        assert step(ctx, p(a), p(lam, 4), p(lam2), None, None) == 1   # lam_next misaligned
        assert step(ctx, p(a), p(lam), p(lam2, 8), None, None) == 1   # lam_out misaligned
        assert step(ctx, p(a), p(lam), p(lam2), p(gF, 2), None) == 1  # dJ/dF misaligned
        assert step(ctx, p(a, 16), p(lam), p(lam2), None, None) == 1  # state off 256 B
        assert step(ctx, None, p(lam), p(lam2), None, None) == 1
        assert seed(ctx, None, p(lam, 4), None, None) == 1
        assert seed(ctx, None, p(lam), p(gF, 2), None) == 1
        assert msd(ctx, None, None, None, p(lam, 8), None, None) == 1
        assert msd(ctx, None, None, p(gF, 2), p(lam), None, None) == 1
        # lbm_step_into: same or overlapping state buffers, or one off 256 B
        assert lib.lbm_step_into(ctx, p(a), p(a), None) == 1
        assert lib.lbm_step_into(ctx, p(a), p(a, 256), None) == 1
        assert lib.lbm_step_into(ctx, p(a), p(b, 128), None) == 1
        # good arguments (dJ/dF at a 4-byte offset is allowed)
        assert step(ctx, p(a), p(lam), p(lam2), p(gF, 4), None) == 0
        assert seed(ctx, None, p(lam), p(gF, 4), None) == 0
        assert msd(ctx, None, None, None, p(lam), p(gF, 4), None) == 0
        torch.cuda.synchronize()
        assert not lib.lbm_last_cuda_error(ctx)
    finally:
        torch.cuda.synchronize()
        lbm.lbm_destroy(ctx)


@pytest.mark.parametrize("Q", [27, 15])
@pytest.mark.parametrize("shape", [(3, 7, 32), (2, 5, 64), (2, 3, 128), (2, 2, 256)])
def test_adjoint_step_long_rows_matches_oracle(lbm, orc, Q, shape):
    """The two-cell adjoint kernel on periodic grids with rows of 32 to 256
    cells (one to eight rows per block) against the oracle's complex-step
    adjoint, with a force field and dJ/dF accumulated onto a nonzero
    field."""
    rho, u = W.taylor_green(shape, u0=0.05, noise=1e-2, seed=36)
    om = W.random_omegas(Q, seed=37)
    F = f32(W.rng(38).uniform(-1e-3, 1e-3, (3,) + shape))
    lam_next = W.rng(39).standard_normal((Q,) + shape)
    S = lbm.Solver(Q, shape, om, force=F)
    S.init_equilibrium(rho, u)
    f_stored = S.get_state().cpu().numpy()
    ln = to_pitched(S, lam_next)
    lo = S.new_adjoint_field()
    g0 = W.rng(40).standard_normal((3,) + shape)
    gF = torch.as_tensor(g0, dtype=torch.float32, device="cuda").contiguous()
    S.adjoint_step(S.current_buffer(), ln, lo, gF)
    torch.cuda.synchronize()
    gF_want = f32(g0).copy()
    want = orc.adjoint_step(Q, shape, f_stored, F, om, lam_next, gF=gF_want)
    got = S.adjoint_view(lo).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    dF = gF.cpu().numpy() - f32(g0)
    dF_want = gF_want - f32(g0)
    assert np.abs(dF - dF_want).max() <= 1e-5 * np.abs(dF_want).max() + 1e-6


def test_adjoint_step_refuses_overlapping_fields(lbm):
    """The adjoint step reads lam_next at neighbouring cells while it writes
    lam_out, so two fields that share any byte are refused (LBM_EINVAL)
    before anything is launched; fields that only touch are accepted."""
    shape = (4, 6, 8)
    S = lbm.Solver(27, shape, W.omegas(27, 1.2))
    S.init_equilibrium(np.ones(shape), np.zeros((3,) + shape))
    n = lbm.lbm_adjoint_bytes(S.ctx) // 4
    pool = torch.zeros(2 * n + 64, dtype=torch.float32, device="cuda")
    for off in (4, n - 4):  # 16-byte aligned partial overlaps, both directions
        with pytest.raises(lbm.LBMError) as err:
            S.adjoint_step(S.current_buffer(), pool[:n], pool[off:off + n])
        assert err.value.status == 1
        with pytest.raises(lbm.LBMError) as err:
            S.adjoint_step(S.current_buffer(), pool[off:off + n], pool[:n])
        assert err.value.status == 1
    S.adjoint_step(S.current_buffer(), pool[:n], pool[n:2 * n])
    torch.cuda.synchronize()
