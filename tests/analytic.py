"""Closed-form solutions the paper compares against (Sec. 9), plus the
textbook decay of the two-dimensional Taylor-Green vortex."""
import numpy as np


def viscosity(omega_nu):
    """nu = c_s^2 (1/omega_nu - 1/2), c_s^2 = 1/3 (end of Sec. 7)."""
    return (1.0 / omega_nu - 0.5) / 3.0


def plates_profile(z, L, F, nu):
    """Force-driven flow between plates at z = +-L (Sec. 9):
    u(z) = u0 (1 - (z/L)^2), u0 = F L^2 / (2 nu)."""
    return F * L**2 / (2 * nu) * (1.0 - (z / L) ** 2)


def duct_profile(y, z, a, F, nu, rho=1.0, nterms=200):
    """Fully developed flow in a square duct |y|, |z| <= a, Eq. ductFourier:
    u = 16 a^2 F / (rho nu pi^3) sum_n (-1)^(n-1)
        [1 - cosh((2n-1) pi z / 2a) / cosh((2n-1) pi / 2)]
        cos((2n-1) pi y / 2a) / (2n-1)^3."""
    y = np.asarray(y, dtype=float)
    z = np.asarray(z, dtype=float)
    s = np.zeros(np.broadcast(y, z).shape)
    for n in range(1, nterms + 1):
        k = (2 * n - 1) * np.pi / (2 * a)
        # cosh(k z)/cosh(k a) written with exponentials that cannot overflow
        ratio = np.exp(k * (np.abs(z) - a)) * (1 + np.exp(-2 * k * np.abs(z))) / (
            1 + np.exp(-2 * k * a))
        s += (-1) ** (n - 1) * (1 - ratio) * np.cos(k * y) / (2 * n - 1) ** 3
    return 16 * a**2 * F / (rho * nu * np.pi**3) * s


def womersley_profile(z, L, Fm, Omega, nu, t):
    """Flow between plates at z = +-L under F = Fm cos(Omega t): solution of
    du/dt = F + nu u'' with u(+-L) = 0, u = Re[U(z) e^{i Omega t}],
    U = Fm / (i Omega) (1 - cos(beta z / L) / cos(beta)),
    beta = sqrt(-i) Wo, Wo = L sqrt(Omega / nu).  (Sec. 9 prints the
    prefactor as +i Fm / Omega; the equation of motion fixes -i Fm / Omega.)"""
    wo = L * np.sqrt(Omega / nu)
    beta = np.sqrt(-1j) * wo
    U = Fm / (1j * Omega) * (1 - np.cos(beta * z / L) / np.cos(beta))
    return np.real(U * np.exp(1j * Omega * t))


def taylor_green_energy_ratio(nu, kx, ky, t):
    """Kinetic energy of the 2D Taylor-Green vortex relative to t = 0:
    exp(-2 nu (kx^2 + ky^2) t)."""
    return np.exp(-2 * nu * (kx**2 + ky**2) * t)
