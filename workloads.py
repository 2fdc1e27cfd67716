"""Seeded synthetic inputs shared by the tests, the bench and the smoke run.

This module only draws numbers and lays out fields: it holds none of the
lattice Boltzmann arithmetic (no equilibria, no moments, no collision).  The
CUDA path and the FP64 oracle each turn these fields into distributions with
their own code.  Every generator is numpy's PCG64 with an explicit seed, so
both sides receive bit-identical FP64 arrays.

Field layout: scalars [nz, ny, nx], vectors [3, nz, ny, nx]; cell (i, j, k)
sits at x = i, y = j, z = k (0-based cell centres), and k_L = 2 pi / N.
"""
from __future__ import annotations

import numpy as np

SEED_NOISE = 20120206      # velocity noise of the Taylor-Green workloads
SEED_FORCE = 20120207      # body-force field of the adjoint workload
SEED_FD_CELLS = 20120208   # finite-difference sample cells
SEED_STATES = 20120209     # random non-equilibrium states of the unit tests


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def taylor_green(shape, u0=0.02, noise=0.0, seed=SEED_NOISE, two_d=False):
    """Density 1 and the Taylor-Green velocity
        u =  u0 sin(k x) cos(k y) cos(k z)
        v = -u0 cos(k x) sin(k y) cos(k z),   w = 0
    (the z factor is dropped for the z-invariant 2D vortex), plus iid uniform
    noise in [-noise, noise] on every component.  shape = (nz, ny, nx)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky, kz = 2 * np.pi / nx, 2 * np.pi / ny, 2 * np.pi / nz
    cz = np.ones(shape) if two_d else np.cos(kz * z)
    u = np.zeros((3,) + tuple(shape))
    u[0] = u0 * np.sin(kx * x) * np.cos(ky * y) * cz
    u[1] = -u0 * np.cos(kx * x) * np.sin(ky * y) * cz
    if noise:
        u += rng(seed).uniform(-noise, noise, size=u.shape)
    return np.ones(shape), u


def gaussian_force_field(shape, rms=1e-5, sigma=4.0, seed=SEED_FORCE):
    """Per-component N(0,1) white noise, smoothed by a periodic Gaussian
    filter of standard deviation ``sigma`` cells (FFT), scaled to ``rms``."""
    r = rng(seed)
    F = r.standard_normal((3,) + tuple(shape))
    ks = [np.fft.fftfreq(n) * 2 * np.pi for n in shape]
    kz, ky, kx = np.meshgrid(*ks, indexing="ij")
    filt = np.exp(-0.5 * sigma**2 * (kx**2 + ky**2 + kz**2))
    for c in range(3):
        F[c] = np.real(np.fft.ifftn(np.fft.fftn(F[c]) * filt))
    F *= rms / np.sqrt(np.mean(F**2))
    return F


def random_states(n, Q, seed=SEED_STATES, spread=0.5):
    """n strongly non-equilibrium cells: f_alpha = (1 + spread*U(-1,1)) / Q,
    cell-major [n, Q]."""
    return (1.0 + spread * rng(seed).uniform(-1.0, 1.0, size=(n, Q))) / Q


def random_field_state(shape, Q, seed=SEED_STATES, spread=0.5):
    """A random state [Q, nz, ny, nx] (same recipe as ``random_states``)."""
    return (1.0 + spread * rng(seed).uniform(-1.0, 1.0, size=(Q,) + tuple(shape))) / Q


def random_forces(n, scale=1e-2, seed=SEED_STATES + 1):
    """n body forces, each component U(-scale, scale), [n, 3]."""
    return rng(seed).uniform(-scale, scale, size=(n, 3))


def random_omegas(Q, lo=0.3, hi=1.9, seed=SEED_STATES + 2):
    """Q relaxation rates, distinct, U(lo, hi); entries 0..3 unused."""
    om = rng(seed).uniform(lo, hi, size=Q)
    om[:4] = 0.0
    return om


def omegas(Q, omega_nu, others=1.0):
    """Relaxation rates of the paper's tests: omega_4..omega_8 = omega_nu
    (shear viscosity nu = (1/omega_nu - 1/2)/3), all others ``others``."""
    om = np.full(Q, float(others))
    om[:4] = 0.0
    om[4:9] = omega_nu
    return om


def sample_cells(shape, count, seed=SEED_FD_CELLS):
    """``count`` distinct flat cell indices of a grid, sorted."""
    N = int(np.prod(shape))
    return np.sort(rng(seed).choice(N, size=min(count, N), replace=False))
