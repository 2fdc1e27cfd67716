"""Validation problems of the paper's Sec. 9 on the GPU path: the plates
sweep across the stated Reynolds numbers, the grid-convergence study under
diffusive scaling, and Womersley flow under a time-periodic force (with
oracle parity of the time-dependent forcing).

Geometry: the paper's N nodes across the channel include the two wall
nodes; with half-way bounce-back the N - 2 fluid cells sit between walls
half a cell outside them, L = (N - 2) / 2 (this reproduces the stated Wo
and, within about 1 %, the stated Re)."""
import numpy as np
import pytest

import analytic
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


def plates_steady(lbm, Q, N, omega_nu, Fx, sr32=False):
    """Steady force-driven flow between plates: 3 x 3 x (N - 2) fluid cells,
    walls on the z faces; returns (z, u_x(z), u_analytic(z), nu, L).
    sr32: the stochastically rounded FP32 update (LBM_F32_SR)."""
    nz = N - 2
    shape = (nz, 3, 3)
    L = nz / 2
    nu = analytic.viscosity(omega_nu)
    S = lbm.Solver(Q, shape, W.omegas(Q, omega_nu), force=(Fx, 0.0, 0.0), walls=lbm.LBM_WALL_Z,
                   sr32=sr32)
    S.init_equilibrium(np.ones(shape), np.zeros((3,) + shape))
    # the slowest mode decays as exp(-nu (pi / 2L)^2 t): run to e^-16
    steps = int(16 * 4 * L * L / (nu * np.pi**2)) + 1
    S.step(steps)
    _, u = S.macroscopic()
    ux = u[0].double().mean(dim=(1, 2)).cpu().numpy()
    z = np.arange(nz) + 0.5 - L
    return z, ux, analytic.plates_profile(z, L, Fx, nu), nu, L


@pytest.mark.parametrize("Q,omega_nu,Fx,Re", [
    (15, 1.818, 2e-7, 3.6), (15, 1.818, 4e-7, 7.2), (15, 1.818, 6e-7, 10.7),
    (27, 1.818, 2e-7, 3.6), (27, 1.818, 4e-7, 7.2), (27, 1.818, 6e-7, 10.7),
    (15, 1.923, 1e-6, 111.8), (15, 1.961, 1e-6, 447.2)])
def test_plates_sweep_reynolds_numbers(lbm, Q, omega_nu, Fx, Re):
    """Sec. 9 plates, 3 x 3 x 45 nodes: the steady profile matches
    u0 (1 - (z/L)^2); the centre-line Reynolds number u_max L / nu matches the
    closed form F L^3 / (2 nu^2) and, within the paper's rounding and its
    unstated conventions (about 1 %), the value it states (3.6, 7.2, 10.7 at
    omega 1.818; 111.8, 447.2 at 1.923, 1.961)."""
    z, ux, ua, nu, L = plates_steady(lbm, Q, 45, omega_nu, Fx)
    err = np.linalg.norm(ux - ua) / np.linalg.norm(ua)
    re = ux.max() * L / nu
    re_exact = ua.max() * L / nu
    print("D3Q%d omega %.3f F %.1e: Re %.2f (closed form %.2f, paper %.1f), rel L2 %.2e" % (
        Q, omega_nu, Fx, re, re_exact, Re, err))
    assert err <= 1e-2
    assert re == pytest.approx(re_exact, rel=1e-2)
    assert re == pytest.approx(Re, rel=2e-2)


def _oracle_plates_error(orc, Q, N, omega_nu, Fx):
    nz = N - 2
    L = nz / 2
    shape = (nz, 1, 1)
    nu = analytic.viscosity(omega_nu)
    F = np.array([np.float32(Fx), 0.0, 0.0])
    f = orc.equilibrium(Q, np.ones(shape), np.zeros((3,) + shape), F)
    steps = int(16 * 4 * L * L / (nu * np.pi**2)) + 1
    f = orc.run(Q, shape, f, F, W.omegas(Q, omega_nu), steps, bc=orc.WALL_Z)
    _, u = orc.macroscopic(Q, f, F)
    z = np.arange(nz) + 0.5 - L
    ua = analytic.plates_profile(z, L, Fx, nu)
    return np.linalg.norm(u[0, :, 0, 0] - ua) / np.linalg.norm(ua)


def test_grid_convergence_matches_fp64(lbm, orc):
    """Sec. 9 convergence study (D3Q15, 3 x 3 x N, omega 1.818, F_x = 6.958e-6
    at N = 13 scaled as 1/L^3, diffusive scaling), N = 13, 25, 49, 97.  With
    the stochastically rounded FP32 update (LBM_F32_SR) the GPU errors equal
    the FP64 oracle's at N = 13, 25 and fall with a log-log slope in
    [-2.1, -1.9] against L (the paper reports -1.96; the oracle's -2.0 is
    pinned in test_oracle_pins).  The default round-to-nearest update is
    printed beside it: at steady state it makes the same rounding error at
    every step, and on the finest grids (where the scaled force per step is
    1e-8) those errors, accumulated in the slowest mode, leave it off the
    second-order line; it is held only to 1e-3."""
    L13 = (13 - 2) / 2
    Ls, errs = [], []
    for N in (13, 25, 49, 97):
        L = (N - 2) / 2
        Fx = 6.958e-6 * (L13 / L) ** 3
        _, ux, ua, _, _ = plates_steady(lbm, 15, N, 1.818, Fx, sr32=True)
        err = np.linalg.norm(ux - ua) / np.linalg.norm(ua)
        _, ux_rn, _, _, _ = plates_steady(lbm, 15, N, 1.818, Fx)
        err_rn = np.linalg.norm(ux_rn - ua) / np.linalg.norm(ua)
        line = "N %d: F %.3e, rel L2 error %.4e (round-to-nearest update %.4e)" % (N, Fx, err,
                                                                                 err_rn)
        if N <= 25:
            want = _oracle_plates_error(orc, 15, N, 1.818, Fx)
            print(line + ", FP64 oracle %.4e" % want)
            assert err == pytest.approx(want, rel=1e-2)
            assert err_rn == pytest.approx(want, rel=1e-2)
        else:
            print(line)
            assert err_rn <= 1e-3
        Ls.append(L)
        errs.append(err)
    slope = np.polyfit(np.log(Ls), np.log(errs), 1)[0]
    print("log-log slope of the error against L: %.3f" % slope)
    assert -2.1 <= slope <= -1.9


def _womersley_run(lbm, Q, omega_nu, steps, T=10000, Fm=1e-5, sample_every=None, u0=None):
    nz = 43
    shape = (nz, 3, 3)
    S = lbm.Solver(Q, shape, W.omegas(Q, omega_nu), walls=lbm.LBM_WALL_Z)
    u = np.zeros((3,) + shape)
    if u0 is not None:
        u[0] = u0[:, None, None]
    S.set_force((Fm, 0.0, 0.0))
    S.init_equilibrium(np.ones(shape), u)
    Om = 2 * np.pi / T
    out = {}
    for n in range(steps):
        S.set_force((Fm * np.cos(Om * n), 0.0, 0.0))
        S.step(1)
        if sample_every and (n + 1) % sample_every == 0:
            S.set_force((Fm * np.cos(Om * (n + 1)), 0.0, 0.0))
            _, u = S.macroscopic()
            out[n + 1] = u[0].double().mean(dim=(1, 2)).cpu().numpy()
    return S, out


def test_womersley_time_dependent_force_matches_oracle(lbm, orc):
    """The force changes every step (F = F_m cos(Omega t)); the GPU state after
    300 steps matches the FP64 oracle stepped with the same forces."""
    for Q in (15, 27):
        T, Fm, om_nu = 200, 1e-3, 1.724
        S, _ = _womersley_run(lbm, Q, om_nu, 300, T=T, Fm=Fm)
        torch.cuda.synchronize()
        f_gpu = S.get_state().cpu().numpy()
        shape = (43, 3, 3)
        # the GPU run starts from f^at - S(F(0))/2 with F(0) = F_m
        f = orc.equilibrium(Q, np.ones(shape), np.zeros((3,) + shape),
                            np.array([np.float32(Fm), 0.0, 0.0]))
        om = W.omegas(Q, om_nu)
        Om = 2 * np.pi / T
        for n in range(300):
            Fn = np.array([np.float32(Fm * np.cos(Om * n)), 0.0, 0.0])
            f = orc.run(Q, shape, f, Fn, om, 1, bc=orc.WALL_Z)
        w = orc.equilibrium(Q, np.ones((1, 1, 1)), np.zeros((3, 1, 1, 1)), np.zeros(3))
        err = np.linalg.norm(f_gpu - f) / np.linalg.norm(f - w)
        assert err <= 1e-5, (Q, err)


@pytest.mark.parametrize("omega_nu,Wo", [(1.724, 3.3), (1.923, 6.6)])
def test_womersley_profiles_match_analytic(lbm, omega_nu, Wo):
    """Sec. 9 Womersley flow (D3Q15, 3 x 3 x 45 nodes, F_m = 1e-5,
    T = 10000), started from the analytic profile at t = 0: over the second
    period the profiles at eight phases match Re[U(z) e^{i Omega t}]
    (prefactor -i F_m / Omega), and the Womersley number L sqrt(Omega / nu)
    is the stated one."""
    T = 10000
    L = 43 / 2
    nu = analytic.viscosity(omega_nu)
    Om = 2 * np.pi / T
    assert L * np.sqrt(Om / nu) == pytest.approx(Wo, abs=0.05)
    z = np.arange(43) + 0.5 - L
    u_start = analytic.womersley_profile(z, L, 1e-5, Om, nu, 0)
    _, prof = _womersley_run(lbm, 15, omega_nu, 2 * T, T=T, sample_every=T // 8, u0=u_start)
    errs = []
    scale = max(np.abs(analytic.womersley_profile(z, L, 1e-5, Om, nu, t)).max()
                for t in range(T, 2 * T, T // 8))
    for t, ux in sorted(prof.items()):
        if t <= T:
            continue
        ua = analytic.womersley_profile(z, L, 1e-5, Om, nu, t)
        errs.append(np.abs(ux - ua).max() / scale)
    print("Wo %.1f: max error / max |u| over the period: %.2e" % (Wo, max(errs)))
    assert max(errs) <= 1e-2


def _duct_steady(lbm, Q, omega_nu, Fx, n=43):
    shape = (n, n, 3)
    a = n / 2
    nu = analytic.viscosity(omega_nu)
    S = lbm.Solver(Q, shape, W.omegas(Q, omega_nu), force=(Fx, 0.0, 0.0), walls=3)
    S.init_equilibrium(np.ones(shape), np.zeros((3,) + shape))
    # slowest mode decays as exp(-2 nu (pi / 2a)^2 t): run to e^-12
    steps = int(12 / (2 * nu * (np.pi / (2 * a)) ** 2)) + 1
    S.step(steps)
    _, u = S.macroscopic()
    ux = u[0].double().mean(dim=2).cpu().numpy()  # [z, y]
    c = np.arange(n) + 0.5 - a
    Z, Y = np.meshgrid(c, c, indexing="ij")
    ua = analytic.duct_profile(Y, Z, a, Fx, nu)
    err = np.linalg.norm(ux - ua) / np.linalg.norm(ua)
    return err, ux.max() * a / nu, steps


@pytest.mark.parametrize("Q,omega_nu", [(27, 1.923), (15, 1.818)])
def test_paper_square_duct_re_65_7(lbm, Q, omega_nu):
    """Sec. 9 square duct: 3 x 45 x 45 nodes (43 x 43 fluid cells, a = 21.5),
    centre-line Reynolds number u_max a / nu = 65.7, run to steady state:
    u_x(y, z) matches the series of Eq. ductFourier within 2e-2 (relative L2)
    and Re matches 65.7 within 2 % (the coarse grid and tau = 0.52 put the
    computed profile about 1 % below the series).  D3Q27 runs the stated parameters
    (F_x = 1e-6, omega_nu = 1.923).  D3Q15 is unstable at that omega for a
    flow in the y-z plane (see the next test), so it runs the same Reynolds
    number at omega_nu = 1.818 with the force scaled to match
    (F_x = Re nu / (a u_max(F = 1)))."""
    a = 43 / 2
    nu = analytic.viscosity(omega_nu)
    Fx = 65.7 * nu / (a * analytic.duct_profile(0.0, 0.0, a, 1.0, nu))
    err, re, steps = _duct_steady(lbm, Q, omega_nu, Fx)
    print("D3Q%d square duct, omega %.3f, F %.3e, %d steps: rel L2 %.2e, Re %.2f" % (
        Q, omega_nu, Fx, steps, err, re))
    assert err <= 2e-2
    assert re == pytest.approx(65.7, rel=2e-2)


def test_d3q15_duct_instability_is_reported(lbm):
    """D3Q15 on the duct at omega_nu = 1.923 (the paper's parameters) grows a
    density mode and overflows within a few thousand steps -- in the FP64
    oracle as well (stable up to omega_nu = 1.85, unstable from 1.88; any
    flow in the y-z plane does this, the walls are not the cause; D3Q27
    stays stable up to 1.961).  The library reports the overflowed state as
    LBM_ENONFINITE from the FP64 conservation sums, without any GPU fault,
    and the context stays usable."""
    import ctypes
    n = 43
    shape = (n, n, 3)
    S = lbm.Solver(15, shape, W.omegas(15, 1.923), force=(1e-6, 0.0, 0.0), walls=3)
    S.init_equilibrium(np.ones(shape), np.zeros((3,) + shape))
    S.step(6000)
    out = (ctypes.c_double * 4)()
    assert lbm.load().lbm_conservation(S.ctx, out, None) == 5  # LBM_ENONFINITE
    S.set_omega(W.omegas(15, 1.818))
    S.init_equilibrium(np.ones(shape), np.zeros((3,) + shape))
    S.step(3000)
    assert np.isfinite(S.conservation()).all()


@pytest.mark.parametrize("Q", [27, 15])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_taylor_green_2d_decay_matches_closed_form(lbm, Q, storage):
    """z-invariant 2D Taylor-Green vortex (the closed-form case of the 32^3 flow) at
    128^2, omega_nu = 1.9 (nu = 0.0088), beyond the oracle's reach: between
    steps 500 and 2500 the kinetic energy decays at 2 nu (kx^2 + ky^2)
    within 2.5e-3 (the O(k^2) lattice error is -1.2e-3), for FP32 and
    stochastically rounded FP16 storage."""
    N = 128
    shape = (1, N, N)
    nu = analytic.viscosity(1.9)
    rho, u = W.taylor_green(shape, u0=0.02, two_d=True)
    S = lbm.Solver(Q, shape, W.omegas(Q, 1.9), storage=storage)
    S.init_equilibrium(rho, u)
    S.step(500)
    e0 = S.kinetic_energy()
    S.step(2000)
    e1 = S.kinetic_energy()
    k = 2 * np.pi / N
    rate = np.log(e0 / e1) / 2000
    print("D3Q%d %s: decay rate / closed form - 1 = %.2e" % (Q, storage,
                                                             rate / (4 * nu * k * k) - 1))
    assert abs(rate / (2 * nu * 2 * k * k) - 1) < 2.5e-3
