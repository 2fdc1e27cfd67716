"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test holds it against a
printed table or formula of the paper, an invariant, a closed form, or a
brute-force evaluation, chosen so that a dropped term, a wrong sign or index,
or a transposed operand anywhere in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

import analytic
import paper_printed as pp
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# k_beta of the printed kernels (Sec. 7; App. G): g_beta = omega_beta / k_beta [...]
K_BETA = {
    27: [12, 12, 12, 12, 36, 18, 24, 24, 24, 8, 8, 8, 8, 12, 24, 8, 8, 8, 8, 8, 8, 8, 8],
    15: [8, 8, 8, 4, 12, 18, 16, 16, 16, 8, 16],
}


def _state(Q, n=257, seed=7):
    f = W.random_states(n, Q, seed=seed)
    F = W.random_forces(n, scale=1e-2, seed=seed + 1)
    om = W.random_omegas(Q, seed=seed + 2)
    return f, F, om


def _central_monomials(f, u, e, powers):
    """Brute force: sum_alpha f_alpha prod_i (e_alpha,i - u_i)^p_i."""
    d = e[None, :, :] - u[:, None, :]
    return np.stack([np.sum(f * d[:, :, 0] ** m * d[:, :, 1] ** n * d[:, :, 2] ** p, axis=1)
                     for (m, n, p) in powers], axis=1)


POW27 = [(m, n, p) for m in range(3) for n in range(3) for p in range(3)]


@pytest.mark.parametrize("Q,fname", [(27, "K_d3q27.txt"), (15, "K_d3q15.txt")])
def test_basis_equals_printed_matrix(oracle_lib, Q, fname):
    """K built from the basis polynomials (Sec. 2 / App. G) equals the matrix
    printed in App. A / App. G, and its columns 1..3 are the velocity set."""
    e, K, D, _ = oracle_lib.lattice(Q)
    Kg = np.loadtxt(os.path.join(GOLDEN, fname))
    assert Kg.shape == (Q, Q)
    np.testing.assert_array_equal(K, Kg)
    np.testing.assert_array_equal(K[:, 1:4], e)
    np.testing.assert_array_equal(K[:, 0], np.ones(Q))


@pytest.mark.parametrize("Q", [27, 15])
def test_basis_orthogonal_and_exact_inverse(oracle_lib, Q):
    """K^T K = D diagonal (orthogonality, Sec. 2), so K^-1 = D^-1 K^T exactly."""
    _, K, D, _ = oracle_lib.lattice(Q)
    G = K.T @ K
    np.testing.assert_array_equal(G, np.diag(np.diag(G)))
    np.testing.assert_array_equal(np.diag(G), D)
    np.testing.assert_allclose(K @ (np.diag(1 / D) @ K.T), np.eye(Q), atol=1e-15)


def test_velocity_sets_are_the_stated_ones(oracle_lib):
    """Eq. velocityd3qq27 / Eq. velocityd3q15: rest, 6 axis, 12 edge, 8 corner
    (D3Q27) and rest, 6 axis, 8 corner (D3Q15), each vector once."""
    e27, _, _, _ = oracle_lib.lattice(27)
    assert sorted(map(tuple, e27)) == sorted(
        (a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
    e15, _, _, _ = oracle_lib.lattice(15)
    norms = sorted(int(v @ v) for v in e15)
    assert norms == [0] + [1] * 6 + [3] * 8
    assert len(set(map(tuple, e15))) == 15


@pytest.mark.parametrize("Q,idx", [(27, pp.IDX27), (15, pp.IDX15)])
def test_index_sets_are_the_monomials(oracle_lib, Q, idx):
    """App. B / App. G: each raw moment's +/- index sets equal the monomial
    e_x^m e_y^n e_z^p over the velocity order used by the oracle."""
    e, _, _, _ = oracle_lib.lattice(Q)
    for key, (A, B) in idx.items():
        m, n, p = key.count("x"), key.count("y"), key.count("z")
        mono = e[:, 0] ** m * e[:, 1] ** n * e[:, 2] ** p
        want = np.zeros(Q, dtype=int)
        want[A] = 1
        want[B] = -1
        np.testing.assert_array_equal(mono, want, err_msg=key)


@pytest.mark.parametrize("Q", [27, 15])
def test_collision_kernel_equals_printed_kernels(oracle_lib, Q):
    """The cascade computed from its definition equals the explicit kernels
    printed in Sec. 7 (D3Q27, seven printed coefficients read as corrected)
    and App. G (D3Q15, as printed), on random non-equilibrium states with
    random forces and distinct relaxation rates."""
    e, _, _, _ = oracle_lib.lattice(Q)
    f, F, om = _state(Q)
    _, g, _ = oracle_lib.collide(Q, f, F, om)
    gp, _ = (pp.kernels_q27 if Q == 27 else pp.kernels_q15)(f, F, om, e)
    np.testing.assert_array_equal(g[:, :4], 0.0)
    scale = np.abs(gp).max(axis=0)
    assert (np.abs(g - gp)[:, 4:] <= 1e-12 * scale[4:]).all()


@pytest.mark.parametrize("Q", [27, 15])
def test_source_projections_equal_printed(oracle_lib, Q):
    """<K_beta|S> of the oracle's source equals the printed m^s of App. D
    (D3Q27) / App. G (D3Q15); on D3Q15 S also equals the printed rows."""
    e, K, _, _ = oracle_lib.lattice(Q)
    f, F, _ = _state(Q)
    rho = f.sum(1)
    u = (f @ e + 0.5 * F) / rho[:, None]
    S = oracle_lib.source(Q, u, F)
    ms = (pp.ms_q27 if Q == 27 else pp.ms_q15)(F, u)
    np.testing.assert_allclose(S @ K, ms, rtol=0, atol=1e-15)
    if Q == 15:
        np.testing.assert_allclose(S, pp.source_q15(ms), rtol=0, atol=1e-16)


def test_d3q27_source_central_moments_are_galilean(oracle_lib):
    """Eq. discretecentralsources: on D3Q27 every central moment of S about u
    vanishes except the first-order ones, which equal F (all 27 monomials,
    brute force)."""
    e, _, _, _ = oracle_lib.lattice(27)
    rng = W.rng(11)
    u = rng.uniform(-0.2, 0.2, (64, 3))
    F = rng.uniform(-0.05, 0.05, (64, 3))
    S = oracle_lib.source(27, u, F)
    c = _central_monomials(S, u, e, POW27)
    for k, (m, n, p) in enumerate(POW27):
        if m + n + p == 1:
            i = [m, n, p].index(1)
            np.testing.assert_allclose(c[:, k], F[:, i], atol=1e-16)
        else:
            np.testing.assert_allclose(c[:, k], 0.0, atol=1e-16)


def test_d3q15_source_first_and_second_moments(oracle_lib):
    """On D3Q15 the source has zero mass, first raw moments F and second
    raw moments sigma'_ij of App. C (its third-order central moments alias)."""
    e, _, _, _ = oracle_lib.lattice(15)
    rng = W.rng(12)
    u = rng.uniform(-0.2, 0.2, (32, 3))
    F = rng.uniform(-0.05, 0.05, (32, 3))
    S = oracle_lib.source(15, u, F)
    np.testing.assert_allclose(S.sum(1), 0.0, atol=5e-17)
    np.testing.assert_allclose(S @ e, F, atol=1e-16)
    sg = pp.raw_source_moments(F, u)
    for key, (i, j) in {"xx": (0, 0), "yy": (1, 1), "zz": (2, 2), "xy": (0, 1),
                        "xz": (0, 2), "yz": (1, 2)}.items():
        np.testing.assert_allclose(S @ (e[:, i] * e[:, j]), sg[key], atol=1e-16)


@pytest.mark.parametrize("Q", [27, 15])
def test_cascade_matrix_triangular_with_printed_diagonal(oracle_lib, Q):
    """A[beta][gamma] = <P_beta(e - u)|K_gamma> is lower triangular for
    beta, gamma >= 4 with diagonal k_beta independent of u, as the printed
    kernels' omega_beta / k_beta prefactors require (Sec. 7, App. F, App. G)."""
    f, F, om = _state(Q, n=64)
    _, _, _, A = oracle_lib.collide(Q, f, F, om, want_A=True)
    sub = A[:, 4:, 4:]
    upper = np.triu(np.ones((Q - 4, Q - 4), dtype=bool), 1)
    assert np.abs(sub[:, upper]).max() < 1e-13
    np.testing.assert_allclose(np.diagonal(sub, axis1=1, axis2=2),
                               np.broadcast_to(K_BETA[Q], (64, Q - 4)), atol=1e-12)


@pytest.mark.parametrize("Q", [27, 15])
def test_collision_conserves_mass_and_adds_force(oracle_lib, Q):
    """g_0..g_3 = 0 and the source: mass is conserved and momentum changes by
    exactly F (Sec. 4, App. F)."""
    e, _, _, _ = oracle_lib.lattice(Q)
    f, F, om = _state(Q)
    out, _, _ = oracle_lib.collide(Q, f, F, om)
    np.testing.assert_allclose(out.sum(1), f.sum(1), atol=4e-16)
    np.testing.assert_allclose(out @ e - f @ e, F, atol=4e-16)


@pytest.mark.parametrize("Q", [27, 15])
def test_relaxation_reaches_attractor_with_unit_rates(oracle_lib, Q):
    """With every omega_beta = 1 and F = 0, the post-collision central moments
    are the attractors of Eq. transformedcentralmomentattractors: rho, 0,
    rho/3 on the diagonal, 0 off it, (rho/3)^2 for xxyy and (rho/3)^3 for
    xxyyzz (D3Q27: all 27 monomials; D3Q15: its relaxed moments)."""
    e, _, _, _ = oracle_lib.lattice(Q)
    f, _, _ = _state(Q, n=40)
    F = np.zeros((40, 3))
    out, _, _ = oracle_lib.collide(Q, f, F, np.ones(Q))
    rho = f.sum(1)
    u = (f @ e) / rho[:, None]
    pw = POW27 if Q == 27 else [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1),
                                (0, 1, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 2, 0), (2, 1, 0),
                                (2, 0, 1), (1, 1, 1), (2, 2, 0)]
    c = _central_monomials(out, u, e, pw)
    for k, (m, n, p) in enumerate(pw):
        evens = all(v % 2 == 0 for v in (m, n, p))
        if (m, n, p) == (0, 0, 0):
            want = rho
        elif evens:
            want = (rho / 3) ** ((m + n + p) // 2)
        else:
            want = 0.0 * rho
        np.testing.assert_allclose(c[:, k], want, atol=2e-15, err_msg=str((m, n, p)))


@pytest.mark.parametrize("Q", [27, 15])
def test_attractor_state_is_a_fixed_point(oracle_lib, Q):
    """A cell at its attractor with zero force is left unchanged by the
    collision for any relaxation rates and any density."""
    rng = W.rng(13)
    rho = rng.uniform(0.8, 1.2, 50)
    u = rng.uniform(-0.1, 0.1, (3, 50))
    feq = oracle_lib.equilibrium(Q, rho, u, np.zeros(3)).T
    out, g, _ = oracle_lib.collide(Q, feq, np.zeros((50, 3)), W.random_omegas(Q, seed=3))
    np.testing.assert_allclose(out, feq, atol=2e-16)
    np.testing.assert_allclose(g, 0.0, atol=2e-16)


@pytest.mark.parametrize("Q", [27, 15])
def test_equilibrium_returns_its_density_and_velocity(oracle_lib, Q):
    """Eqs. densitycalculation, velocitycalculation applied to f^at - S/2
    give back rho and u (the +F/2 shift undoes the -S/2)."""
    rng = W.rng(14)
    shape = (3, 4, 5)
    rho = rng.uniform(0.9, 1.1, shape)
    u = rng.uniform(-0.05, 0.05, (3,) + shape)
    F = rng.uniform(-1e-3, 1e-3, (3,) + shape)
    f = oracle_lib.equilibrium(Q, rho, u, F)
    r2, u2 = oracle_lib.macroscopic(Q, f, F)
    np.testing.assert_allclose(r2, rho, atol=1e-15)
    np.testing.assert_allclose(u2, u, atol=1e-16)


def test_d3q27_equilibrium_product_form_at_unit_density(oracle_lib):
    """At rho = 1 the D3Q27 attractor state factorises into 1D weights
    (2/3 - u^2, (1/3 + u^2 +- u)/2) per axis, and at u = 0 it gives the
    weights 8/27, 2/27, 1/54, 1/216."""
    e, _, _, _ = oracle_lib.lattice(27)
    rng = W.rng(15)
    u = rng.uniform(-0.1, 0.1, (3, 20))
    f = oracle_lib.equilibrium(27, np.ones(20), u, np.zeros(3))

    def w1(c, v):
        return np.where(c == 0, 2 / 3 - v**2, 0.5 * (1 / 3 + v**2 + c * v))

    want = np.stack([w1(e[a, 0], u[0]) * w1(e[a, 1], u[1]) * w1(e[a, 2], u[2])
                     for a in range(27)])
    np.testing.assert_allclose(f, want, atol=1e-16)
    f0 = oracle_lib.equilibrium(27, np.ones(1), np.zeros((3, 1)), np.zeros(3))[:, 0]
    w = {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}
    np.testing.assert_allclose(f0, [w[int(v @ v)] for v in e], atol=1e-17)


@pytest.mark.parametrize("Q", [27, 15])
def test_complex_step_jacobian_matches_differences(oracle_lib, Q):
    """The complex-step Jacobian equals fourth-order central differences."""
    f, F, om = _state(Q, n=3)
    J = oracle_lib.collide_jacobian(Q, f, F, om)
    h = 1e-4
    x0 = np.concatenate([f, F], axis=1)
    Jfd = np.zeros_like(J)
    for k in range(Q + 3):
        outs = []
        for s in (2, 1, -1, -2):
            x = x0.copy()
            x[:, k] += s * h
            outs.append(oracle_lib.collide(Q, x[:, :Q], x[:, Q:], om)[0])
        Jfd[:, :, k] = (-outs[0] + 8 * outs[1] - 8 * outs[2] + outs[3]) / (12 * h)
    np.testing.assert_allclose(J, Jfd, atol=1e-9)


@pytest.mark.parametrize("Q,bc", [(27, 0), (27, 1), (15, 3)])
def test_adjoint_step_is_the_transpose_of_the_linearised_step(oracle_lib, Q, bc):
    """<lam_next, df_next> = <lam, df> + <gF, dF> for the linearisation of
    one collide-and-stream step (central differences), periodic and walled."""
    shape = (5, 3, 4)
    f = W.random_field_state(shape, Q, seed=21, spread=0.3)
    rng = W.rng(22)
    F = rng.uniform(-1e-3, 1e-3, (3,) + shape)
    om = W.random_omegas(Q, seed=23)
    lam_next = rng.standard_normal((Q,) + shape)
    df = rng.standard_normal((Q,) + shape)
    dF = rng.standard_normal((3,) + shape)
    gF = np.zeros((3,) + shape)
    lam = oracle_lib.adjoint_step(Q, shape, f, F, om, lam_next, bc=bc, gF=gF)
    h = 1e-6
    fp = oracle_lib.run(Q, shape, f + h * df, F + h * dF, om, 1, bc=bc)
    fm = oracle_lib.run(Q, shape, f - h * df, F - h * dF, om, 1, bc=bc)
    lhs = np.sum(lam_next * (fp - fm) / (2 * h))
    rhs = np.sum(lam * df) + np.sum(gF * dF)
    assert abs(lhs - rhs) <= 1e-7 * abs(lhs)


@pytest.mark.parametrize("Q", [27, 15])
def test_macroscopic_grad_matches_differences(oracle_lib, Q):
    """The chain rule through Eqs. densitycalculation and velocitycalculation
    (seed of the adjoint for an objective of rho and u) equals central
    differences of J = <g_rho, rho> + <g_u, u> in every population and force
    component, and for J = sum rho |u|^2 / 2 it reduces to the kinetic-energy
    seed u.e - |u|^2 / 2, u / 2."""
    shape = (2, 3, 2)
    rng = W.rng(25)
    f = W.random_field_state(shape, Q, seed=26, spread=0.4)
    F = rng.uniform(-1e-2, 1e-2, (3,) + shape)
    g_rho = rng.standard_normal(shape)
    g_u = rng.standard_normal((3,) + shape)
    dfl, dF = oracle_lib.macroscopic_grad(Q, f, F, g_rho, g_u)

    def J(ff, FF):
        rho, u = oracle_lib.macroscopic(Q, ff, FF)
        return np.sum(g_rho * rho) + np.sum(g_u * u)

    h = 1e-6
    for idx in np.ndindex(f.shape):
        fp, fm = f.copy(), f.copy()
        fp[idx] += h
        fm[idx] -= h
        assert dfl[idx] == pytest.approx((J(fp, F) - J(fm, F)) / (2 * h), rel=1e-7, abs=1e-8)
    for idx in np.ndindex(F.shape):
        Fp, Fm = F.copy(), F.copy()
        Fp[idx] += h
        Fm[idx] -= h
        assert dF[idx] == pytest.approx((J(f, Fp) - J(f, Fm)) / (2 * h), rel=1e-7, abs=1e-8)
    rho, u = oracle_lib.macroscopic(Q, f, F)
    ke_f, ke_F = oracle_lib.kinetic_energy_grad(Q, f, F)
    mg_f, mg_F = oracle_lib.macroscopic_grad(Q, f, F, 0.5 * np.sum(u * u, axis=0), rho * u)
    np.testing.assert_allclose(mg_f, ke_f, atol=1e-14)
    np.testing.assert_allclose(mg_F, ke_F, atol=1e-14)


@pytest.mark.parametrize("Q", [27, 15])
def test_streaming_moves_and_bounces(oracle_lib, Q):
    """Eq. cascadedstreaming1 with a collision that is the identity (all rates
    zero, no force): each population moves one link; at a wall it comes back
    to its own cell reversed (half-way bounce-back)."""
    e, _, _, _ = oracle_lib.lattice(Q)
    shape = (4, 3, 5)
    rng = W.rng(24)
    tag = rng.uniform(0.0, 1.0, (Q,) + shape)
    om = np.zeros(Q)  # every omega_beta = 0 and F = 0: g = 0 and S = 0
    out = oracle_lib.run(Q, shape, tag, np.zeros(3), om, 1, bc=oracle_lib.WALL_Z)
    nz, ny, nx = shape
    for a in range(Q):
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    tz = z + e[a, 2]
                    ty = (y + e[a, 1]) % ny
                    tx = (x + e[a, 0]) % nx
                    if 0 <= tz < nz:
                        assert out[a, tz, ty, tx] == pytest.approx(tag[a, z, y, x], abs=1e-15)
                    else:
                        b = int(np.where((e == -e[a]).all(1))[0][0])
                        assert out[b, z, y, x] == pytest.approx(tag[a, z, y, x], abs=1e-15)


@pytest.mark.parametrize("Q", [27, 15])
def test_force_driven_plates_converge_to_parabola(oracle_lib, Q):
    """Sec. 9, first test: body-force flow between plates with half-way
    bounce-back gives u = u0 (1 - (z/L)^2), u0 = F L^2 / (2 nu); the error
    falls about fourfold when the resolution doubles (second order)."""
    errs = []
    for N in (10, 20):
        shape = (N, 1, 1)
        om = W.omegas(Q, 1.25)
        nu = analytic.viscosity(1.25)
        F = np.array([1e-6, 0.0, 0.0])
        f = oracle_lib.equilibrium(Q, np.ones(shape), np.zeros((3,) + shape), F)
        f = oracle_lib.run(Q, shape, f, F, om, 12 * N * N, bc=oracle_lib.WALL_Z)
        _, u = oracle_lib.macroscopic(Q, f, F)
        z = np.arange(N) + 0.5 - N / 2
        ua = analytic.plates_profile(z, N / 2, 1e-6, nu)
        errs.append(np.linalg.norm(u[0, :, 0, 0] - ua) / np.linalg.norm(ua))
        np.testing.assert_allclose(u[1:], 0.0, atol=1e-15)
    assert errs[1] < (1e-3 if Q == 27 else 6e-3)
    assert 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.slow
@pytest.mark.parametrize("Q", [15, 27])
def test_square_duct_converges_to_series(oracle_lib, Q):
    """Sec. 9, Eq. ductFourier: force-driven flow in a square duct with walls
    on the y and z faces converges to the Fourier series, second order."""
    errs = []
    for N in (8, 16):
        shape = (N, N, 1)
        om = W.omegas(Q, 1.25)
        nu = analytic.viscosity(1.25)
        F = np.array([1e-6, 0.0, 0.0])
        f = oracle_lib.equilibrium(Q, np.ones(shape), np.zeros((3,) + shape), F)
        f = oracle_lib.run(Q, shape, f, F, om, 8 * N * N,
                           bc=oracle_lib.WALL_Y | oracle_lib.WALL_Z)
        _, u = oracle_lib.macroscopic(Q, f, F)
        c = np.arange(N) + 0.5 - N / 2
        Z, Y = np.meshgrid(c, c, indexing="ij")
        ua = analytic.duct_profile(Y, Z, N / 2, 1e-6, nu)
        errs.append(np.linalg.norm(u[0, :, :, 0] - ua) / np.linalg.norm(ua))
    assert errs[1] < (5e-3 if Q == 27 else 2e-2)
    assert 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.parametrize("Q", [27, 15])
def test_taylor_green_2d_decay_rate(oracle_lib, Q):
    """z-invariant 2D Taylor-Green vortex, 32^2, tau = 0.6: after the start-up
    transient the kinetic energy decays at 2 nu (kx^2 + ky^2) to 1e-3."""
    N = 32
    shape = (1, N, N)
    om = W.omegas(Q, 1 / 0.6)
    nu = analytic.viscosity(1 / 0.6)
    rho, u = W.taylor_green(shape, two_d=True)
    f = oracle_lib.equilibrium(Q, rho, u, np.zeros(3))
    energies = []
    for _ in range(2):
        f = oracle_lib.run(Q, shape, f, np.zeros(3), om, 50)
        energies.append(oracle_lib.kinetic_energy(Q, f, np.zeros(3)))
    k = 2 * np.pi / N
    rate = np.log(energies[0] / energies[1]) / 50
    assert abs(rate / (2 * nu * 2 * k * k) - 1) < 1e-3


def test_viscosity_relation():
    """nu = c_s^2 (1/omega - 1/2): tau = 0.6 gives 1/30; omega = 1.818 gives
    about 0.0167 and Re 3.6 for F = 2e-7 and L = 21.5 (Sec. 9)."""
    assert analytic.viscosity(1 / 0.6) == pytest.approx(1 / 30)
    nu = analytic.viscosity(1.818)
    assert nu == pytest.approx(0.0167, abs=1e-4)
    L = 21.5
    u0 = 2e-7 * L**2 / (2 * nu)
    assert u0 * L / nu == pytest.approx(3.6, abs=0.05)


@pytest.mark.slow
def test_grid_convergence_under_diffusive_scaling(oracle_lib):
    """Sec. 9 convergence study: D3Q15 plates, omega 1.818, N = 13, 25, 49
    nodes across (L = (N - 2) / 2), F_x = 6.958e-6 at N = 13 scaled as
    1/L^3.  The relative L2 velocity error is second order: its log-log slope
    against L is -2 (the paper reports -1.96)."""
    Q = 15
    errs, Ls = [], []
    for N in (13, 25, 49):
        nz = N - 2
        L = nz / 2
        shape = (nz, 1, 1)
        nu = analytic.viscosity(1.818)
        Fx = 6.958e-6 * (5.5 / L) ** 3
        F = np.array([Fx, 0.0, 0.0])
        f = oracle_lib.equilibrium(Q, np.ones(shape), np.zeros((3,) + shape), F)
        steps = int(16 * 4 * L * L / (nu * np.pi**2)) + 1
        f = oracle_lib.run(Q, shape, f, F, W.omegas(Q, 1.818), steps, bc=oracle_lib.WALL_Z)
        _, u = oracle_lib.macroscopic(Q, f, F)
        z = np.arange(nz) + 0.5 - L
        ua = analytic.plates_profile(z, L, Fx, nu)
        errs.append(np.linalg.norm(u[0, :, 0, 0] - ua) / np.linalg.norm(ua))
        Ls.append(L)
    slope = np.polyfit(np.log(Ls), np.log(errs), 1)[0]
    assert -2.1 <= slope <= -1.9
